"""CP-ALS serving on one GPU: continuous batching over the library's CP-ALS batch.

``Server.submit`` takes a COO tensor (host arrays) and CP-ALS parameters and
returns a Future. An admission thread encodes requests on its own stream
(alto_encode) as device memory allows: a request is admitted while the
resident bytes of the runs in flight plus its own peak bytes
(alto_cpals_footprint) stay within the budget and a batch slot is free. The
loop thread adds encoded requests to the batch, advances every active run by
one mode update per step (alto_batch_step, a replayed CUDA graph; two steps
per round, up to three rounds queued ahead of the host), polls the
asynchronous state read-backs, and normalises finished runs in place; a
retire thread copies their results (factors, lambda, fits) to the host
(alto_batch_copy_out) and completes the futures, and the loop thread then
frees the slots. Requests that arrive while
others are on the GPU join at the next step, so their work overlaps.

``run_fcfs`` is the one-at-a-time reference: the same library, one request
after the other in arrival order, each encoded and solved with cpals_run.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from concurrent.futures import Future
from typing import List, Optional, Sequence

import numpy as np

from . import AltoError, Batch, alto_cpals_footprint, alto_encode, alto_fill_uniform


@dataclasses.dataclass
class CPResult:
    factors: List[np.ndarray]
    lam: np.ndarray
    fits: List[float]
    iters_done: int
    status: int
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclasses.dataclass
class _Request:
    coords: np.ndarray
    vals: np.ndarray
    dims: tuple
    R: int
    iters: int
    tol: float
    init: List[np.ndarray]
    arrival: float
    future: Future
    peak: int = 0
    resident: int = 0
    tensor: object = None
    admitted: float = 0.0
    seed: int = 0


def device_factors(dims: Sequence[int], R: int, seed: int, stream=None):
    """Initial factors drawn on the GPU: factor m = alto_fill_uniform(seed * 16 + m)."""
    import torch
    out = []
    for m, d in enumerate(dims):
        a = torch.empty((int(d), int(R)), dtype=torch.float32, device="cuda")
        alto_fill_uniform(a, (int(seed) * 16 + m) % (1 << 32), stream)
        out.append(a)
    return out


def percentile(xs: Sequence[float], q: float) -> float:
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


class Server:
    """Continuous-batching CP-ALS server (see module docstring)."""

    def __init__(self, budget_bytes: float = 100e9, max_slots: int = 1024, steps_per_round: int = 2,
                 staging_bytes: int = 256 << 20):
        import torch
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.steps_per_round = int(steps_per_round)
        self.batch = Batch(max_slots=max_slots)
        self.encode_stream = torch.cuda.Stream()
        self._lock = threading.Condition()
        self._waiting: collections.deque = collections.deque()   # submitted, not encoded
        self._ready: collections.deque = collections.deque()     # encoded, not in the batch
        self._live = {}                                          # slot -> request
        self._retiring: list = []                                # (slot, request, iters, status)
        self._resident = 0
        self._admitted = 0
        self._stop = False
        self.latencies: List[float] = []
        self.completed = 0
        self.errors = 0
        self.work_nnz_r_iters = 0.0
        self.t_first: Optional[float] = None
        self.t_last: Optional[float] = None
        # host seconds the loop thread spends per phase, and device time of the steps
        self.loop_s = {"add": 0.0, "step_poll": 0.0, "retire_enqueue": 0.0, "retire_finish": 0.0,
                       "remove": 0.0, "free": 0.0, "batch_add": 0.0}
        self.batch_gpu_ms = 0.0
        self._loop_done = False
        self._to_remove: list = []
        self.retire_stream = torch.cuda.Stream()
        # Page-locked staging for uploads (admission thread) and downloads
        # (retire thread): copies from pageable memory go through the driver's
        # own staging and slow every other thread's CUDA calls meanwhile.
        self._up = torch.empty(staging_bytes, dtype=torch.uint8, pin_memory=True).numpy()
        self._down = torch.empty(staging_bytes, dtype=torch.uint8, pin_memory=True).numpy()
        self._admit_thread = threading.Thread(target=self._admit_loop, daemon=True)
        self._loop_thread = threading.Thread(target=self._loop, daemon=True)
        self._retire_thread = threading.Thread(target=self._retire_loop, daemon=True)
        self._admit_thread.start()
        self._loop_thread.start()
        self._retire_thread.start()

    # -- public --------------------------------------------------------------
    def submit(self, coords: np.ndarray, vals: np.ndarray, dims: Sequence[int], R: int, iters: int,
               init: Optional[Sequence[np.ndarray]] = None, seed: int = 0, tol: float = 0.0,
               arrival: Optional[float] = None) -> Future:
        """``init``: host initial factors, or None to draw them on the GPU from
        ``seed`` (factor m filled by alto_fill_uniform with seed * 16 + m)."""
        fut: Future = Future()
        init_l = None if init is None else [np.ascontiguousarray(a, dtype=np.float32) for a in init]
        req = _Request(np.asarray(coords), np.asarray(vals, dtype=np.float32), tuple(int(d) for d in dims),
                       int(R), int(iters), float(tol), init_l,
                       time.perf_counter() if arrival is None else arrival, fut)
        req.seed = int(seed)
        req.resident, req.peak = alto_cpals_footprint(req.dims, req.vals.shape[0], req.R, req.iters)
        with self._lock:
            if self.t_first is None:
                self.t_first = req.arrival
            self._waiting.append(req)
            self._lock.notify_all()
        return fut

    def close(self, timeout: Optional[float] = None) -> None:
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._admit_thread.join(timeout)
        self._loop_thread.join(timeout)
        self._retire_thread.join(timeout)
        self.batch.sync()
        self.batch_gpu_ms = self.batch.info().gpu_ms
        self.batch.free()

    def stats(self) -> dict:
        span = (self.t_last - self.t_first) if (self.t_first is not None and self.t_last) else float("nan")
        return {"completed": self.completed, "errors": self.errors,
                "batch_gpu_s": self.batch_gpu_ms / 1000.0,
                "gpu_busy_fraction": (self.batch_gpu_ms / 1000.0 / span) if span and span > 0 else float("nan"),
                "loop_host_s": dict(self.loop_s),
                "p50_s": percentile(self.latencies, 50), "p99_s": percentile(self.latencies, 99),
                "mean_s": float(np.mean(self.latencies)) if self.latencies else float("nan"),
                "requests_per_s": self.completed / span if span and span > 0 else float("nan"),
                "nnz_r_iters_per_s": self.work_nnz_r_iters / span if span and span > 0 else float("nan"),
                "makespan_s": span}

    # -- admission thread: encode while memory allows ------------------------
    def _admit_loop(self) -> None:
        import torch
        while True:
            with self._lock:
                while not self._stop and not self._can_admit():
                    self._lock.wait(0.002)
                if self._stop and not self._waiting:
                    return
                if not self._can_admit():
                    continue
                req = self._waiting.popleft()
                self._resident += req.resident
                self._admitted += 1
            try:
                with torch.cuda.stream(self.encode_stream):
                    coords, vals = self._stage_upload(req.coords, req.vals)
                    req.tensor = alto_encode(coords, vals, req.dims, stream=self.encode_stream)
                    Batch.prepare(req.tensor, req.R)  # its waits stay off the loop thread
                    # initial factors on the encode stream (the batch orders
                    # itself after the handle's stream)
                    if req.init is None:
                        req.init = device_factors(req.dims, req.R, req.seed, self.encode_stream)
                    else:
                        req.init = [torch.from_numpy(a).pin_memory().cuda(non_blocking=True)
                                    for a in req.init]
                req.admitted = time.perf_counter()
                with self._lock:
                    self._ready.append(req)
                    self._lock.notify_all()
            except AltoError as e:
                with self._lock:
                    self._resident -= req.resident
                    self._admitted -= 1
                    self.errors += 1
                req.future.set_exception(e)

    def _stage_upload(self, coords: np.ndarray, vals: np.ndarray):
        """The request's COO arrays copied into the pinned upload buffer
        (alto_encode copies them in and waits, so the buffer is free again
        when it returns); arrays that do not fit go as they are."""
        cb = coords.size * 4
        vb = vals.size * 4
        if cb + vb > self._up.size:
            return coords, vals
        c = self._up[:cb].view(np.uint32).reshape(coords.shape)
        v = self._up[cb:cb + vb].view(np.float32)
        np.copyto(c, coords, casting="unsafe")
        np.copyto(v, vals, casting="unsafe")
        return c, v

    def _can_admit(self) -> bool:
        if not self._waiting or self._admitted >= self.max_slots:
            return False
        req = self._waiting[0]
        if self._admitted == 0:
            return True  # always admit one, even over budget
        return self._resident + req.peak <= self.budget

    # -- loop thread: batch steps, polls, retirement -------------------------
    def _loop(self) -> None:
        import torch
        while True:
            with self._lock:
                ready = list(self._ready)
                self._ready.clear()
                idle = not ready and not self._live and not self._to_remove
                if idle:
                    if self._stop and not self._waiting and self._admitted == 0 and not self._retiring:
                        self._loop_done = True
                        self._lock.notify_all()
                        return
                    self._lock.wait(0.002)
                    continue
            t_a = time.perf_counter()
            with self._lock:
                gone = self._to_remove
                self._to_remove = []
            for slot, req in gone:
                t_r = time.perf_counter()
                self.batch.remove(slot)
                t_f = time.perf_counter()
                req.tensor.free()
                req.tensor = None
                self.loop_s["remove"] += t_f - t_r
                self.loop_s["free"] += time.perf_counter() - t_f
            t_ba = time.perf_counter()
            for req in ready:
                try:
                    slot = self.batch.add(req.tensor, req.R, req.iters, req.init, tol=req.tol)
                    self._live[slot] = req
                except AltoError as e:
                    self._finish_error(req, e)
            t_b = time.perf_counter()
            self.loop_s["add"] += t_b - t_a
            self.loop_s["batch_add"] += t_b - t_ba
            if self._live:
                self.batch.step(self.steps_per_round)
                done = self.batch.poll(wait=False)
                info = self.batch.info()
                self.batch_gpu_ms = info.gpu_ms
                if not done and info.pending_readbacks >= 3:  # keep ~3 rounds queued on the GPU
                    done = self.batch.poll(wait=True)
                t_c = time.perf_counter()
                self.loop_s["step_poll"] += t_c - t_b
                for slot in done:
                    req = self._live.pop(slot)
                    # normalise in place; the retire thread copies the slot
                    # out (alto_batch_copy_out) and hands it back for removal
                    iters_done, status = self.batch.result(slot, [None] * len(req.dims))
                    with self._lock:
                        self._retiring.append((slot, req, iters_done, status))
                        self._lock.notify_all()
                self.loop_s["retire_enqueue"] += time.perf_counter() - t_c
            elif not ready:
                with self._lock:
                    self._lock.wait(0.001)

    # -- retire thread: copy results out, finish the futures -----------------
    def _retire_loop(self) -> None:
        import torch
        while True:
            with self._lock:
                while not self._retiring and not (self._stop and self._loop_done):
                    self._lock.wait(0.002)
                if not self._retiring:
                    return
                item = self._retiring.pop(0)
            t0 = time.perf_counter()
            slot, req, iters_done, status = item
            res_f = self._download(slot, req)
            now = time.perf_counter()
            res_f, lam_h, fits_h = res_f
            res = CPResult(res_f, lam_h, fits_h[:iters_done].tolist(), iters_done, status, req.arrival,
                           req.admitted, now)
            with self._lock:
                self._to_remove.append((slot, req))
                self._resident -= req.resident
                self._admitted -= 1
                self.completed += 1
                self.latencies.append(res.latency)
                self.work_nnz_r_iters += float(req.vals.shape[0]) * req.R * iters_done
                self.t_last = now
                self.loop_s["retire_finish"] += now - t0
                self._lock.notify_all()
            req.future.set_result(res)

    def _download(self, slot: int, req: _Request):
        """The slot's factors, lambda and fits through the pinned download
        buffer (one factor at a time when they do not fit together)."""
        N = len(req.dims)
        sizes = [d * req.R * 4 for d in req.dims]
        small = 8 * req.R + 8 * req.iters
        lam_h = np.empty(req.R)
        fits_h = np.zeros(req.iters)
        out = [np.empty((d, req.R), dtype=np.float32) for d in req.dims]
        if sum(sizes) + small <= self._down.size:
            offs = np.cumsum([0] + sizes)
            bufs = [self._down[offs[m]:offs[m + 1]].view(np.float32) for m in range(N)]
            lb = self._down[offs[N]:offs[N] + 8 * req.R].view(np.float64)
            fb = self._down[offs[N] + 8 * req.R:offs[N] + small].view(np.float64)
            self.batch.copy_out(slot, bufs, lb, fb, stream=self.retire_stream)
            for m in range(N):
                np.copyto(out[m].reshape(-1), bufs[m])
            np.copyto(lam_h, lb)
            np.copyto(fits_h, fb)
        else:
            for m in range(N):
                if sizes[m] <= self._down.size:
                    buf = self._down[:sizes[m]].view(np.float32)
                    self.batch.copy_out(slot, [buf if k == m else None for k in range(N)],
                                        stream=self.retire_stream)
                    np.copyto(out[m].reshape(-1), buf)
                else:
                    self.batch.copy_out(slot, [out[m] if k == m else None for k in range(N)],
                                        stream=self.retire_stream)
            lb = self._down[:8 * req.R].view(np.float64)
            fb = self._down[8 * req.R:small].view(np.float64)
            self.batch.copy_out(slot, [None] * N, lb, fb, stream=self.retire_stream)
            np.copyto(lam_h, lb)
            np.copyto(fits_h, fb)
        return out, lam_h, fits_h

    def _finish_error(self, req: _Request, e: Exception) -> None:
        if req.tensor is not None:
            req.tensor.free()
        with self._lock:
            self._resident -= req.resident
            self._admitted -= 1
            self.errors += 1
            self._lock.notify_all()
        req.future.set_exception(e)


def run_fcfs(requests, schedule_start: float) -> dict:
    """One-at-a-time reference: each request, in arrival order and no earlier
    than its arrival, encoded and solved alone with cpals_run (ungrouped
    launches, no graphs), its factors copied back to the host. ``requests``
    yields (arrival_offset_s, coords, vals, dims, R, iters, init, seed), init
    None for factors drawn on the GPU as the Server does. Returns latency /
    throughput statistics."""
    import torch
    lat, work = [], 0.0
    not_spd = 0
    t_first = t_last = None
    # the same pinned staging the Server uses
    up = torch.empty(256 << 20, dtype=torch.uint8, pin_memory=True).numpy()
    down = torch.empty(256 << 20, dtype=torch.uint8, pin_memory=True)
    for arrival_off, coords, vals, dims, R, iters, init, seed in requests:
        arrival = schedule_start + arrival_off
        now = time.perf_counter()
        if now < arrival:
            time.sleep(arrival - now)
        if t_first is None:
            t_first = arrival
        cb, vb = coords.size * 4, vals.size * 4
        if cb + vb <= up.size:
            c = up[:cb].view(np.uint32).reshape(coords.shape)
            v = up[cb:cb + vb].view(np.float32)
            np.copyto(c, coords, casting="unsafe")
            np.copyto(v, vals, casting="unsafe")
            t = alto_encode(c, v, dims)
        else:
            t = alto_encode(coords, vals, dims)
        if init is None:
            A = device_factors(dims, R, seed)
        else:
            A = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in init]
        try:
            lam, fits = t.cpals(R, iters, A)
        except AltoError as e:
            if e.status != -6:  # NOT_SPD ends a run early with its last factors
                raise
            not_spd += 1
            fits = []
        outs = []  # results on the host, through pinned staging as the Server does
        for a in A:
            n = a.numel()
            if n * 4 <= down.numel():
                buf = down[: n * 4].view(torch.float32)
                buf.copy_(a.reshape(-1))
                outs.append(buf.numpy().reshape(a.shape).copy())
            else:
                outs.append(a.cpu().numpy())
        t.free()
        t_last = time.perf_counter()
        lat.append(t_last - arrival)
        work += float(len(vals)) * R * len(fits)
    span = (t_last - t_first) if t_first is not None else float("nan")
    return {"completed": len(lat), "not_spd": not_spd,
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "mean_s": float(np.mean(lat)) if lat else float("nan"),
            "requests_per_s": len(lat) / span if span > 0 else float("nan"),
            "nnz_r_iters_per_s": work / span if span > 0 else float("nan"), "makespan_s": span}
