#!/usr/bin/env python
"""Benchmark: ALTO encode + CP-ALS (10 iterations) on the 10M x 2M x 50k,
100M-nonzero Zipf(1.1) tensor at rank 32, on one GB300 per process.

One step = one pass of the whole hot path over the tensor: encode (bit plan,
linearization, radix sort, partition, hot rows) followed by CP-ALS with 10
iterations (per mode: MTTKRP, Gram, fp64 solve, normalisation; fit per
iteration), starting from the same seeded factors every step.

value = MTTKRP work of the step (iterations x modes x nnz x R) / step time,
summed over ranks (replicas: every rank runs its own copy of the workload).

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MTTKRP nnz*R/s & HBM GB/s vs peak; served CP-ALS p50/p99 vs one-at-a-time"
UNIT = "nnz*R/s"
ITERS = 10
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--nnz", type=int, default=0, help="override nonzeros (testing only)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true", help="skip the served CP-ALS workload")
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-pool", type=int, default=64)
    p.add_argument("--serve-slow-requests", type=int, default=300,
                   help="requests of the second serving run below saturation (0: none)")
    p.add_argument("--serve-slow-rate", type=float, default=25.0,
                   help="arrival rate of that run (requests/s)")
    p.add_argument("--no-cpapr", action="store_true", help="skip the CP-APR measurement")
    p.add_argument("--cpapr-nnz", type=int, default=0, help="override the count tensor's nonzeros")
    p.add_argument("--no-tune", action="store_true",
                   help="library default plans instead of the autotuned ones")
    p.add_argument("--plans", default="",
                   help="per-mode plans 'variant:cols_per_lane,...' instead of tuning (profiling)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the per-mode MTTKRP measurements of the other workloads")
    p.add_argument("--configs-scale", type=float, default=1.0,
                   help="scale the nonzeros of the other workloads (testing only)")
    p.add_argument("--profile-mttkrp", default="",
                   choices=["", "uniform3d", "zipf3d", "count4d", "zipf5d"],
                   help="profiling aid: encode this workload (--nnz scales it), run one MTTKRP "
                        "per mode with --plans (default plans if none) and exit")
    return p.parse_args()


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """Slowest rank's time (the job finishes when the last replica does)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(work_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: every replica's work over the slowest time."""
    return world * work_per_rank / (ms_max / 1000.0)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload(args):
    import synth
    spec = synth.ZIPF3D  # 10M x 2M x 50k, 1e8 nonzeros, Zipf 1.1, R = 32
    if args.nnz:
        spec = synth.scaled(spec, args.nnz)
    return spec


def config_json(spec, extra=None):
    c = {"workload": f"encode + CP-ALS {ITERS} iters: {spec.name}",
         "dims": list(spec.dims), "nnz": spec.nnz, "rank": spec.rank,
         "coords": "Zipf s=1.1 per mode (rank->index permuted)", "values": "lognormal(0,1) fp32",
         "cp_als_iters": ITERS,
         "l2": "inputs larger than L2 (1.6 GB nonzero stream per step)"}
    if extra:
        c.update(extra)
    return c


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


PROFILE_OF_KERNEL = {"mttkrp_kernel": "mttkrp_zipf3d_10Mx2Mx50k_r32.md",
                     "mttkrp_out_kernel": "mttkrp_out_zipf3d_10Mx2Mx50k_r32.md"}


def traffic_from_profiles(kernel_src_sha, kernel="mttkrp_kernel"):
    """dram bytes per launch of the MTTKRP kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if kernel not in PROFILE_OF_KERNEL:
        return None
    path = os.path.join(ROOT, "profiles", PROFILE_OF_KERNEL[kernel])
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_src_sha:
        return None
    return float(t.group(1))


def kernel_src_sha():
    h = hashlib.sha256()
    for f in ("mttkrp.cu", "mttkrp.cuh", "mttkrp_kernel.cuh", "alto_internal.cuh", "outorder.cuh",
              "out_n3.cu"):
        with open(os.path.join(ROOT, "paper_2403_06348_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def algorithmic_bytes_per_mode(coords, dims, R, key_bytes, fbytes=4):
    """M*(key+value bytes) + sum_{m!=n} D_m*R*fbytes + I_n*R*4, D_m = distinct
    rows of mode m (the roofline model of one mode-n MTTKRP)."""
    M = coords.shape[1]
    D = [int(np.count_nonzero(np.bincount(coords[m], minlength=dims[m]))) for m in range(len(dims))]
    out = []
    for n in range(len(dims)):
        b = M * (key_bytes + 4) + sum(D[m] * R * fbytes for m in range(len(dims)) if m != n)
        b += dims[n] * R * 4
        out.append(b)
    return out, D


# ---------------------------------------------------------------------------
# Per-mode MTTKRP measurements of every workload (configs 1-4)
# ---------------------------------------------------------------------------

VARIANT_NAMES = {0: "AUTO", 1: "ATOMIC", 2: "PULL", 3: "OUTPUT", 4: "TILED", 5: "TILED_LINE"}


def time_modes(h, Ad, R, dims, reps=5):
    """Per mode: average MTTKRP launch time (ms; the library's CUDA events on
    the launching stream around the MTTKRP kernels, output zeroing excluded)
    over ``reps`` calls after one warm-up call, and the resolved plan."""
    import torch
    out = torch.empty((max(dims), R), dtype=torch.float32, device="cuda")
    res = []
    for n in range(len(dims)):
        o = out[:dims[n]]
        h.mttkrp(n, Ad, R, out=o)
        torch.cuda.synchronize()
        h.profile_enable(True)
        h.profile_read(reset=True)
        for _ in range(reps):
            h.mttkrp(n, Ad, R, out=o)
        torch.cuda.synchronize()
        pr = h.profile_read(reset=True)
        launches, ms = pr["mttkrp"]
        zms = pr.get("zero", (0, 0.0))[1]
        h.profile_enable(False)
        res.append((ms / max(reps, 1), h.get_mode_plan(n, R), zms / max(reps, 1)))
    del out
    return res


def sampled_error(h, coords, vals, dims, A, Ad, R, nhot=64, nrand=64, seed=11):
    """Max row-relative error of every mode's MTTKRP against the fp64 oracle
    (oracle/coo_ref.c on the original fp32 factors) on sampled rows: the
    nhot most frequent rows and nrand random rows of each mode."""
    import torch
    from oracle import alto_ref as ar
    from oracle import cref
    rng = np.random.default_rng(seed)
    worst = []
    for n in range(len(dims)):
        got = h.mttkrp(n, Ad, R)
        counts = np.bincount(coords[n], minlength=dims[n])
        hot = np.argsort(-counts, kind="stable")[:nhot]
        rnd = rng.choice(dims[n], size=min(nrand, dims[n]), replace=False)
        rows = np.unique(np.concatenate([hot, rnd])).astype(np.uint32)
        ref = cref.mttkrp_rows(coords, vals, dims, A, n, rows)
        g = got[torch.from_numpy(rows.astype(np.int64)).cuda()].cpu().numpy()
        err, bad = ar.row_relative_error(g, ref)
        worst.append(float(err) if bad == 0 else float("inf"))
        del got
    return worst


def config_entry(spec, coords, dims, R, kw, timed, fbytes, peak):
    bytes_mode, _ = algorithmic_bytes_per_mode(coords, dims, R, 8 * kw, fbytes)
    M = coords.shape[1]
    modes = []
    for n, (ms, plan, zms) in enumerate(timed):
        gbs = bytes_mode[n] / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        modes.append({"mode": n, "rows": int(dims[n]), "plan": VARIANT_NAMES.get(plan[0], plan[0]),
                      "cols_per_lane": plan[1], "staged_rows": plan[2], "ms": ms, "zeroing_ms": zms,
                      "nnz_r_per_s": M * R / (ms / 1e3) if ms > 0 else None,
                      "algorithmic_bytes": bytes_mode[n], "gbs": gbs, "frac": gbs / peak})
    tot_ms = sum(m["ms"] for m in modes)
    return {"modes": modes, "all_modes_ms": tot_ms,
            "nnz_r_per_s_all_modes": len(dims) * M * R / (tot_ms / 1e3) if tot_ms > 0 else None,
            "mean_frac": sum(m["frac"] for m in modes) / len(modes)}


def run_configs(args, alto, peak, headline=None):
    """Per-mode MTTKRP of the four single-tensor workloads with autotuned plans
    (configs 1, 3 and 4; config 4 with fp32 and with bf16 factors and its
    error against the fp64 oracle), and the one-copy plans on the headline
    tensor (TILED and ATOMIC: no stored order)."""
    import torch
    import synth
    out = {"method": ("per mode: mean of 5 MTTKRP calls after one warm-up, CUDA events on the "
                      "launching stream around the MTTKRP kernels (zeroing excluded); plans from "
                      "alto_autotune unless named; frac = algorithmic bytes / time / peak")}

    def load(spec):
        if args.configs_scale != 1.0:
            spec = synth.scaled(spec, max(1000, int(spec.nnz * args.configs_scale)))
        c, v = synth.cached(spec)
        return spec, np.asarray(c), np.asarray(v)

    def tuned(spec, coords, vals, R, bf16=False, keep=False):
        dims = spec.dims
        h = alto.alto_encode(torch.from_numpy(coords.view(np.int32)).cuda(), torch.from_numpy(vals).cuda(),
                             dims)
        A = synth.factors(dims, R, seed=1)
        Ad = [torch.from_numpy(a).cuda() for a in A]
        if bf16:
            Ad = [a.to(torch.bfloat16) for a in Ad]
        h.autotune(Ad, R, segments=False, output=True)
        timed = time_modes(h, Ad, R, dims)
        kw = int(h.query().key_words)
        return h, A, Ad, timed, kw

    # config 1: 1000 x 800 x 600, 1e5 distinct uniform nonzeros, R = 16 (launch-bound)
    spec, coords, vals = load(synth.UNIFORM3D)
    h, A, Ad, timed, kw = tuned(spec, coords, vals, spec.rank)
    e = config_entry(spec, coords, spec.dims, spec.rank, kw, timed, 4, peak)
    e["workload"] = spec.name
    e["bound"] = "launch latency (1.35 MB per mode)"
    out["uniform3d_1e5"] = e
    h.free()

    # the headline tensor on the one-copy plans (no stored order)
    if headline is not None:
        spec, coords, vals = headline
        h = alto.alto_encode(torch.from_numpy(coords.view(np.int32)).cuda(), torch.from_numpy(vals).cuda(),
                             spec.dims)
        Ad = [torch.from_numpy(a).cuda() for a in synth.factors(spec.dims, spec.rank, seed=1)]
        kw = int(h.query().key_words)
        one_copy = {}
        for variant, cpl in ((4, 8), (4, 4), (1, 4)):
            for n in range(len(spec.dims)):
                h.set_mode_plan(n, variant, cpl)
            timed = time_modes(h, Ad, spec.rank, spec.dims)
            one_copy[f"{VARIANT_NAMES[variant]}:{cpl}"] = config_entry(spec, coords, spec.dims, spec.rank,
                                                                       kw, timed, 4, peak)
        best = min(one_copy, key=lambda k: one_copy[k]["all_modes_ms"])
        out["zipf3d_1e8_one_copy"] = {"workload": spec.name, "plans": one_copy, "best": best}
        h.free()

    # config 3: 4-mode count tensor, 2e8 nonzeros, R = 16, every mode autotuned
    spec, coords, vals = load(synth.COUNT4D)
    h, A, Ad, timed, kw = tuned(spec, coords, vals, spec.rank)
    e = config_entry(spec, coords, spec.dims, spec.rank, kw, timed, 4, peak)
    e["workload"] = spec.name
    out["count4d_2e8"] = e
    h.free()
    del coords, vals

    # config 4: 5-mode Zipf tensor, 1.5e8 nonzeros, 128-bit positions, R = 64,
    # fp32 and bf16 factors, error against the fp64 oracle on sampled rows
    spec, coords, vals = load(synth.ZIPF5D)
    for bf16 in (False, True):
        h, A, Ad, timed, kw = tuned(spec, coords, vals, spec.rank, bf16=bf16)
        e = config_entry(spec, coords, spec.dims, spec.rank, kw, timed, 2 if bf16 else 4, peak)
        e["workload"] = spec.name + (" bf16 factors" if bf16 else " fp32 factors")
        e["max_row_rel_err_vs_fp64_oracle"] = sampled_error(h, coords, vals, spec.dims, A, Ad, spec.rank)
        e["error_sample"] = "64 most frequent + 64 random rows per mode"
        out["zipf5d_1.5e8_" + ("bf16" if bf16 else "fp32")] = e
        h.free()
    return out


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def host_cpu():
    """The host CPU as the OS reports it (model name or, on Arm, the part)."""
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model", "CPU part"):
        m = re.search(r"^%s\s*:\s*(.+)$" % key, txt, flags=re.M)
        if m:
            return f"{key}: {m.group(1).strip()}"
    return "unknown"


def oracle_sample(coords, vals, dims, R, sample_nnz, threads, modes):
    """The oracle as it stands on the first sample_nnz nonzeros: encode, then
    the Alg. 1 mode updates listed in ``modes`` (C fp64 MTTKRP on ``threads``
    threads). Returns (MTTKRP work nnz*R per second of the whole sample,
    seconds, per-part seconds)."""
    from oracle import alto_ref as ar
    from oracle import cref
    import synth
    c = np.ascontiguousarray(coords[:, :sample_nnz])
    v = np.ascontiguousarray(vals[:sample_nnz])
    A = [a.astype(np.float64) for a in synth.factors(dims, R, seed=7)]
    mk = lambda cc, vv, F, n: cref.mttkrp(cc, vv, dims, F, n, nthreads=threads)
    t0 = time.perf_counter()
    ar.encode(c, v, dims)
    parts = {"encode_s": time.perf_counter() - t0}
    for n in modes:
        t = time.perf_counter()
        ar.cp_als_mode_update(c, v, A, n, mk)
        parts[f"mode{n}_s"] = time.perf_counter() - t
    secs = time.perf_counter() - t0
    return len(modes) * sample_nnz * R / secs, secs, parts


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    spec = workload(args)
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    threads = os.cpu_count() or 1
    sample = min(spec.nnz, 1_000_000)
    N = len(spec.dims)
    work = 0.0
    t_all = 0.0
    for i in range(args.warmup + args.steps):
        rate, secs, _ = oracle_sample(coords, vals, spec.dims, spec.rank, sample, threads, [i % N])
        if i >= args.warmup:
            work += rate * secs
            t_all += secs
    value = work / t_all
    sample_desc = (f"each step: oracle encode + one Alg. 1 mode update (modes in turn; C fp64 "
                   f"MTTKRP on {threads} threads) on the first {sample} of {spec.nnz} "
                   f"nonzeros, dims unchanged; value = MTTKRP nnz*R / time over the timed steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "higher_is_better": True, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / max(args.steps, 1),
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(spec),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu": host_cpu(), "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import paper_2403_06348_gb300 as alto
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    alto.build()
    spec = workload(args)
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    dims, R, M, N = spec.dims, spec.rank, spec.nnz, len(spec.dims)

    coords_d = torch.from_numpy(coords.view(np.int32)).cuda()
    vals_d = torch.from_numpy(vals).cuda()
    A0 = synth.factors(dims, R, seed=1)
    A0d = [torch.from_numpy(a).cuda() for a in A0]
    work = [torch.empty_like(a) for a in A0d]

    # the per-mode plan, measured once on this workload before timing (the
    # autotuner with the stored-order candidates, the default segment count)
    plans = None
    if args.plans:
        plans = [(int(v), int(c), 0 if int(v) == 3 else -1)
                 for v, c in (x.split(":") for x in args.plans.split(","))]
    elif not args.no_tune:
        h = alto.alto_encode(coords_d, vals_d, dims)
        out = torch.empty((max(dims), R), dtype=torch.float32, device="cuda")
        rep = h.autotune(A0d, R, out=out, segments=False, output=True)
        plans = rep["plans"]
        del out
        h.free()

    def step(profile_into=None):
        h = alto.alto_encode(coords_d, vals_d, dims)
        if plans is not None:
            for n, (variant, cpl, hot) in enumerate(plans):
                h.set_mode_plan(n, variant, cpl, hot)
        if profile_into is not None:
            h.profile_enable(True)
        for w, a in zip(work, A0d):
            w.copy_(a)
        lam, fits = h.cpals(R, ITERS, work)
        if profile_into is not None:
            for k, (n, ms) in h.profile_read().items():
                a, b = profile_into.get(k, (0, 0.0))
                profile_into[k] = (a + n, b + ms)
        if profile_into is not None:
            info = h.query()
            enc = profile_into.setdefault("_encode", [0.0, 0.0, 0])
            enc[0] += info.encode_ms
            enc[1] += info.sort_ms
            enc[2] = int(info.sort_passes)
            if "_kw" not in profile_into:
                profile_into["_kw"] = int(info.key_words)
                profile_into["_plans"] = [h.get_mode_plan(n, R) for n in range(N)]
        h.free()
        return fits

    for _ in range(args.warmup):
        fits = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    prof = {}
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = alto.alto_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        fits = step(prof)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    launches = alto.alto_kernel_launches() - launches0
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    work_units = ITERS * N * M * R
    value = job_value(work_units, world, ms)

    # roofline of the dominant kernel (the MTTKRP segment kernel)
    kw = prof.get("_kw", 1)
    used = prof.get("_plans") or []
    outorder = [len(used) > n and used[n][0] == 3 for n in range(N)]
    # the roofline model's bytes: the nonzero stream once, the distinct input
    # rows once, the output once; the same for every plan (a plan's extra
    # traffic, such as a stored order, is overhead, not algorithmic bytes)
    bytes_per_mode, distinct = algorithmic_bytes_per_mode(coords, dims, R, 8 * kw)
    kernel = ("mttkrp_out_kernel" if all(outorder) else
              "mttkrp_kernel" if not any(outorder) else "mttkrp_out_kernel + mttkrp_kernel")
    n_mttkrp, ms_mttkrp = prof.get("mttkrp", (0, 0.0))
    avg_ms = ms_mttkrp / max(n_mttkrp, 1)
    # the output rows are counted as written once; the separate zeroing
    # launch writes every one of them, so the fraction with it is also given
    avg_ms_zero = (ms_mttkrp + prof.get("zero", (0, 0.0))[1]) / max(n_mttkrp, 1)
    avg_bytes = sum(bytes_per_mode) / N
    achieved = avg_bytes / (avg_ms / 1000.0) / 1e9 if avg_ms > 0 else 0.0
    peak, peak_src = measured_peaks()
    sha = kernel_src_sha()
    traffic = traffic_from_profiles(sha, kernel)
    breakdown = {k: {"launches": v[0], "ms_per_step": v[1] / args.steps}
                 for k, v in prof.items() if not k.startswith("_")}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": config_json(spec, {"parallelism": f"replicas x{world}",
                                         "mode_plans": prof.get("_plans")}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "kernel": kernel,
                         "peak_source": f"{peak_src} hbm_gbs",
                         "algorithmic_bytes_per_launch": avg_bytes,
                         "avg_launch_ms": avg_ms, "launches": n_mttkrp,
                         "frac_incl_output_zeroing": (avg_bytes / (avg_ms_zero / 1e3) / 1e9 / peak
                                                      if avg_ms_zero > 0 else None),
                         "source_sha": sha},
            "gpu_launches": launches,
            "clocks": clocks,
            "breakdown_ms_per_step": breakdown,
            "encode": encode_line(prof, M, kw, args.steps, peak),
            "final_fit": fits[-1] if fits else None}

    if not args.no_e2e:
        line["e2e"] = run_e2e(args, alto, coords, vals, spec, A0, world, barrier, plans)
    if not args.no_configs and world == 1:
        line["configs"] = run_configs(args, alto, peak, headline=(spec, coords, vals))
    if not args.no_serve:
        line["serving"] = run_serving(args, alto)
    if not args.no_cpapr and world == 1:
        line["cpapr"] = run_cpapr(args, alto)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        sample = min(M, 2_000_000)
        rate, secs, parts = oracle_sample(coords, vals, dims, R, sample, threads, list(range(N)))
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "cpu": host_cpu(),
                                "sample": (f"oracle encode + one CP-ALS iteration (all {N} mode "
                                           f"updates, C fp64 MTTKRP) on the first {sample} of {M} "
                                           f"nonzeros, dims unchanged: {secs:.1f} s; "
                                           + ", ".join(f"{k} {v:.2f}" for k, v in parts.items()))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _gen_request(r):
    import synth
    return synth.request_tensor(r)


def run_serving(args, alto):
    """Served CP-ALS: Poisson arrivals (200 requests/s) of CP-ALS requests
    (20 iterations; 3-5 modes, dims log-uniform 100..1M, nnz log-uniform
    1e3..1e7, Zipf(1.1) coordinates, values U(0,1], R in {8,16,32}), through
    the continuous-batching Server and, on the same schedule, one request at a
    time (FCFS, cpals_run). Requests carry host COO data; factors are drawn on
    the GPU from the request's seed and come back to pinned host memory.
    Latency = results on the host - arrival."""
    import concurrent.futures
    import multiprocessing
    import threading
    import synth
    from paper_2403_06348_gb300 import serve

    pool, reqs = synth.request_pool_stream(count=args.serve_requests, pool=args.serve_pool)
    t0 = time.perf_counter()
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                                mp_context=ctx) as ex:
        tensors = list(ex.map(_gen_request, pool))
    gen_s = time.perf_counter() - t0
    items = [(r.arrival_s, tensors[r.rid][0], tensors[r.rid][1], r.dims, r.rank, r.iters, None,
              r.seed % (1 << 27)) for r in reqs]
    # warm-up: one small request through each arm
    small = min(range(len(pool)), key=lambda j: pool[j].nnz)
    w = (0.0, tensors[small][0], tensors[small][1], pool[small].dims, 8, 2, None, 1)
    srv = serve.Server(budget_bytes=100e9)
    srv.submit(w[1], w[2], w[3], w[4], w[5], seed=w[7]).result(timeout=120)
    srv.close()
    serve.run_fcfs([w], time.perf_counter())

    def serve_stream(stream):
        srv = serve.Server(budget_bytes=100e9)
        start = time.perf_counter() + 0.05
        futs = []

        def producer():
            for it in stream:
                at = start + it[0]
                now = time.perf_counter()
                if now < at:
                    time.sleep(at - now)
                futs.append(srv.submit(it[1], it[2], it[3], it[4], it[5], seed=it[7], arrival=at))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        results = [f.result(timeout=3600) for f in futs]
        srv.close()
        return srv.stats(), results

    served, results = serve_stream(items)
    fcfs = serve.run_fcfs(items, time.perf_counter() + 0.05)
    nnz = [len(it[2]) for it in items]
    out = {"workload": (f"{len(items)} CP-ALS requests (20 iters), Poisson 200/s, 3-5 modes, dims "
                        f"log-U[100,1M], nnz log-U[1e3,1e7] (pool of {len(pool)} tensors, "
                        f"mean nnz {np.mean(nnz):.3g}), Zipf 1.1, R in {{8,16,32}}, 100 GB budget"),
           "served": served, "one_at_a_time": fcfs,
           "throughput_ratio": served["nnz_r_iters_per_s"] / fcfs["nnz_r_iters_per_s"],
           "p99_ratio": fcfs["p99_s"] / served["p99_s"],
           "not_spd": sum(1 for r in results if r.status != 0),
           "generate_s": gen_s}
    # Both arms are past saturation at 200/s, so their latencies there are
    # mostly queueing. The same requests at a rate below the one-at-a-time
    # arm's capacity give the latency of the work itself.
    if args.serve_slow_requests > 0:
        k = min(args.serve_slow_requests, len(items))
        f = 200.0 / args.serve_slow_rate
        slow = [(it[0] * f,) + tuple(it[1:]) for it in items[:k]]
        s_served, s_results = serve_stream(slow)
        s_fcfs = serve.run_fcfs(slow, time.perf_counter() + 0.05)
        out["below_saturation"] = {
            "workload": f"the first {k} requests of the stream at {args.serve_slow_rate:g}/s (arrivals scaled)",
            "served": s_served, "one_at_a_time": s_fcfs,
            "p50_ratio": s_fcfs["p50_s"] / s_served["p50_s"], "p99_ratio": s_fcfs["p99_s"] / s_served["p99_s"],
            "not_spd": sum(1 for r in s_results if r.status != 0)}
    return out


def run_cpapr(args, alto):
    """CP-APR (multiplicative updates, Alg. 2) on the 4-mode count tensor
    1M x 500k x 200 x 24 (2e8 nonzeros, Zipf 1.2 / uniform, Poisson(3)+1), R = 16:
    two outer iterations, l_max = 10; the Phi launches (Alg. 5) timed with CUDA
    events inside the library."""
    import torch
    import synth
    spec = synth.COUNT4D
    if args.cpapr_nnz:
        spec = synth.scaled(spec, args.cpapr_nnz)
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    R, N, M = spec.rank, len(spec.dims), spec.nnz
    h = alto.alto_encode(torch.from_numpy(coords.view(np.int32)).cuda(), torch.from_numpy(vals).cuda(),
                         spec.dims)
    init = [(0.1 + a).astype(np.float32) for a in synth.factors(spec.dims, R, seed=3)]
    A = [torch.from_numpy(a).cuda() for a in init]
    h.cpapr(R, [a.clone() for a in A], k_max=1, l_max=1)  # warm-up
    h.profile_enable(True)
    h.profile_read(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = h.cpapr(R, A, k_max=2)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    n_phi, ms_phi = h.profile_read()["mttkrp"]
    h.free()
    # a mode's inner loop evaluates Phi once per step plus the final check;
    # the launches after convergence return at once (counted in ms_phi)
    evaluated = sum(min(10, st + 1) for row in rep["inner"] for st in row)
    per = ms_phi / max(evaluated, 1)
    return {"workload": f"CP-APR MU, {spec.name}, R={R}, k_max=2, l_max=10",
            "seconds": secs, "outer_done": rep["outer_done"], "inner_steps": rep["inner"],
            "pre_modes": rep["pre_modes"], "objective": rep["objective"],
            "phi_launches": n_phi, "phi_evaluations": evaluated, "phi_ms_per_evaluation": per,
            "phi_nnz_r_per_s": M * R / (per / 1000.0) if evaluated else None}


def run_e2e(args, alto, coords, vals, spec, A0, world, barrier, plans=None):
    """Same step through the C ABI with pinned HOST buffers: the library copies
    coords/values/factors in and the factors, lambda and fits out."""
    import torch
    dims, R, M, N = spec.dims, spec.rank, spec.nnz, len(spec.dims)
    ch = torch.from_numpy(coords.view(np.int32)).pin_memory()
    vh = torch.from_numpy(vals).pin_memory()
    Ah = [torch.from_numpy(a).pin_memory() for a in A0]
    work = [torch.empty_like(a).pin_memory() for a in Ah]
    cn, vn = ch.numpy(), vh.numpy()
    wn = [w.numpy() for w in work]

    def step():
        h = alto.alto_encode(cn, vn, dims)
        if plans is not None:
            for n, (variant, cpl, hot) in enumerate(plans):
                h.set_mode_plan(n, variant, cpl, hot)
        h.cpals(R, ITERS, wn)
        h.free()

    def reset():  # the initial factors again (cpals_run overwrites them); not timed
        for w, a in zip(work, Ah):
            w.copy_(a)

    reset()
    step()
    steps = max(1, min(args.steps, 3))
    total = 0.0
    for _ in range(steps):
        reset()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()  # host COO in, host factors in and out: every copy is inside
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
    ms = max_over_ranks(total / steps * 1000.0, world)
    h2d = coords.nbytes + vals.nbytes + sum(a.nbytes for a in A0)
    d2h = sum(a.nbytes for a in A0) + 8 * R + 8 * ITERS
    return {"value": job_value(ITERS * N * M * R, world, ms), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ms,
            "steps": steps}


def encode_line(prof, M, kw, steps, peak):
    """The encode's device time per step and the radix sort's bandwidth: per
    8-bit pass the positions and values are read and written once, and the
    digit counts of all passes take one more read of the positions."""
    enc_ms, sort_ms, passes = prof.get("_encode", [0.0, 0.0, 0])
    enc_ms, sort_ms = enc_ms / steps, sort_ms / steps
    sort_bytes = M * passes * (2 * 8 * kw + 2 * 4) + M * 8 * kw
    gbs = sort_bytes / (sort_ms / 1e3) / 1e9 if sort_ms > 0 else 0.0
    return {"ms_per_step": enc_ms, "sort_ms": sort_ms, "sort_passes": passes,
            "sort_bytes": sort_bytes, "sort_gbs": gbs, "sort_frac": gbs / peak,
            "bytes_model": "M*(passes*(2*8*kw + 2*4) + 8*kw): positions and values read "
                           "and written once per pass, plus one read for the digit counts"}


def run_profile_mttkrp(args):
    """One MTTKRP per mode of a named workload, for an ncu capture of the
    MTTKRP kernels alone (no tuning launches before them)."""
    import torch
    import paper_2403_06348_gb300 as alto
    import synth
    spec = {"uniform3d": synth.UNIFORM3D, "zipf3d": synth.ZIPF3D, "count4d": synth.COUNT4D,
            "zipf5d": synth.ZIPF5D}[args.profile_mttkrp]
    if args.nnz:
        spec = synth.scaled(spec, args.nnz)
    alto.build()
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    h = alto.alto_encode(torch.from_numpy(coords.view(np.int32)).cuda(), torch.from_numpy(vals).cuda(),
                         spec.dims)
    R = spec.rank
    A = [torch.from_numpy(a).cuda() for a in synth.factors(spec.dims, R, seed=1)]
    plans = [tuple(int(v) for v in x.split(":")) for x in args.plans.split(",")] if args.plans else []
    out = torch.empty((max(spec.dims), R), dtype=torch.float32, device="cuda")
    for n in range(len(spec.dims)):
        if n < len(plans):
            h.set_mode_plan(n, plans[n][0], plans[n][1])
        h.mttkrp(n, A, R, out=out[:spec.dims[n]])
    torch.cuda.synchronize()
    print(json.dumps({"workload": spec.name, "plans": [h.get_mode_plan(n, R) for n in range(len(spec.dims))]}))
    h.free()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_mttkrp:
        return run_profile_mttkrp(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
