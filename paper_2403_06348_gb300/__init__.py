"""Python binding of libalto (ALTO sparse tensors on GB300, sm_103a).

Thin ctypes marshalling over the C ABI in include/alto.h: every step of the
encode, MTTKRP and CP-ALS path runs in the library's CUDA kernels. PyTorch is
used only for device memory and streams. There is no CPU fallback: if the
compiled library is missing, ``lib()`` raises.

The module-level functions carry the C names (``alto_encode``,
``alto_mttkrp``, ``cpals_run``, ...); ``AltoTensor`` wraps a handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# ALTO_LIB points the binding at another build of the library (e.g. a tuning
# variant); by default the in-tree build is used.
LIB_PATH = os.environ.get("ALTO_LIB") or os.path.join(_PKG, "_build", "libalto.so")

ALTO_MAX_MODES = 8
ALTO_MAX_HOT = 4096
ALTO_F32, ALTO_BF16 = 0, 1
VARIANT_AUTO, VARIANT_ATOMIC, VARIANT_PULL, VARIANT_OUTPUT = 0, 1, 2, 3
VARIANT_TILED, VARIANT_TILED_LINE = 4, 5

STATUS_NAMES = {0: "ALTO_OK", -1: "ALTO_ERR_INVALID_ARG", -2: "ALTO_ERR_OOM", -3: "ALTO_ERR_CUDA",
                -4: "ALTO_ERR_UNSUPPORTED", -5: "ALTO_ERR_COORD_RANGE", -6: "ALTO_ERR_NOT_SPD",
                -7: "ALTO_ERR_TIMEOUT"}


class AltoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class alto_allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                           ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.c_void_p)),
                ("ctx", ctypes.c_void_p)]


class alto_info(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int), ("nbits", ctypes.c_int), ("key_words", ctypes.c_int),
                ("status", ctypes.c_int), ("nnz", ctypes.c_uint64), ("nparts", ctypes.c_uint64),
                ("dims", ctypes.c_uint64 * ALTO_MAX_MODES), ("bits", ctypes.c_int * ALTO_MAX_MODES),
                ("mask_lo", ctypes.c_uint64 * ALTO_MAX_MODES),
                ("mask_hi", ctypes.c_uint64 * ALTO_MAX_MODES),
                ("max_interval", ctypes.c_uint32 * ALTO_MAX_MODES),
                ("nhot", ctypes.c_uint32 * ALTO_MAX_MODES), ("norm_sq", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("encode_ms", ctypes.c_float),
                ("sort_ms", ctypes.c_float), ("sort_passes", ctypes.c_int)]


PROF_KINDS = ("mttkrp", "pull_reduce", "zero", "gram", "solve", "rmul", "pos_out")


class alto_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * len(PROF_KINDS)),
                ("ms", ctypes.c_double * len(PROF_KINDS))]


class alto_mode_plan(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("cols_per_lane", ctypes.c_int),
                ("hot_rows", ctypes.c_int)]


class alto_tune_result(ctypes.Structure):
    _fields_ = [("plan", alto_mode_plan * ALTO_MAX_MODES), ("ms", ctypes.c_double * ALTO_MAX_MODES),
                ("default_ms", ctypes.c_double * ALTO_MAX_MODES), ("nparts", ctypes.c_uint64),
                ("candidates", ctypes.c_int)]


ALTO_TUNE_SEGMENTS = 1
ALTO_TUNE_OUTPUT = 2


class alto_apr_params(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int), ("l_max", ctypes.c_int), ("tau", ctypes.c_double),
                ("kappa", ctypes.c_double), ("kappa_tol", ctypes.c_double), ("eps", ctypes.c_double),
                ("variant", ctypes.c_int)]


class alto_apr_stats(ctypes.Structure):
    _fields_ = [("outer_done", ctypes.c_int), ("converged", ctypes.c_int),
                ("inner_steps_total", ctypes.c_int), ("pre_modes", ctypes.c_int)]


APR_AUTO, APR_OTF, APR_PRE = 0, 1, 2


class alto_batch_info(ctypes.Structure):
    _fields_ = [("active", ctypes.c_int), ("slots_span", ctypes.c_int), ("steps", ctypes.c_uint64),
                ("graph_launches", ctypes.c_uint64), ("bytes_held", ctypes.c_uint64),
                ("pending_readbacks", ctypes.c_int), ("gpu_ms", ctypes.c_double)]


# Exported symbols and their ctypes signatures (mirrors include/alto.h).
_vp, _u64, _i32, _u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
SIGNATURES = {
    "alto_encode": ([_vp, _vp, _vp, _i32, _u64, _vp, _vp, _vp], _i32),
    "alto_free": ([_vp], None),
    "alto_query": ([_vp, ctypes.POINTER(alto_info)], _i32),
    "alto_set_partitions": ([_vp, _u64, _vp], _i32),
    "alto_copy_partition": ([_vp, _vp, _vp], _i32),
    "alto_copy_encoded": ([_vp, _vp, _vp, _vp], _i32),
    "alto_decode": ([_vp, _vp, _vp, _vp], _i32),
    "alto_copy_hot_rows": ([_vp, _i32, _vp, _u32, ctypes.POINTER(_u32)], _i32),
    "alto_set_mode_plan": ([_vp, _i32, ctypes.POINTER(alto_mode_plan)], _i32),
    "alto_get_mode_plan": ([_vp, _i32, _i32, ctypes.POINTER(alto_mode_plan)], _i32),
    "alto_build_pos_out": ([_vp, _i32, _u64, _vp], _i32),
    "alto_copy_pos_out": ([_vp, _i32, _vp, ctypes.POINTER(_u64), _vp], _i32),
    "alto_free_pos_out": ([_vp, _i32], _i32),
    "alto_mttkrp": ([_vp, _i32, _vp, _i32, _i32, _vp, _vp], _i32),
    "cpals_run": ([_vp, _i32, _i32, _vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(_i32), _vp],
                  _i32),
    "alto_mttkrp_noalloc": ([_vp, _i32, _vp, _i32, _i32, _vp, _vp], _i32),
    "alto_mttkrp_grouped": ([_i32, _vp, _vp, _vp, _vp, _i32, _vp, _vp], _i32),
    "alto_batch_create": ([_i32, _vp, _vp, ctypes.POINTER(_vp)], _i32),
    "alto_batch_free": ([_vp], None),
    "alto_batch_add": ([_vp, _vp, _i32, _i32, ctypes.c_double, _vp, ctypes.POINTER(_i32)], _i32),
    "alto_batch_prepare": ([_vp, _i32], _i32),
    "alto_batch_step": ([_vp, _i32], _i32),
    "alto_batch_poll": ([_vp, _i32, _vp, _i32, ctypes.POINTER(_i32)], _i32),
    "alto_batch_result": ([_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
                          _i32),
    "alto_batch_copy_out": ([_vp, _i32, _vp, _vp, _vp, _vp], _i32),
    "alto_batch_remove": ([_vp, _i32], _i32),
    "alto_batch_query": ([_vp, ctypes.POINTER(alto_batch_info)], _i32),
    "alto_batch_sync": ([_vp], _i32),
    "alto_cpals_footprint": ([_i32, _vp, _u64, _i32, _i32, ctypes.POINTER(_u64),
                              ctypes.POINTER(_u64)], _i32),
    "alto_fill_uniform": ([_vp, _u64, _u64, _vp], _i32),
    "alto_phi": ([_vp, _i32, _vp, _vp, _i32, ctypes.c_double, _i32, _vp, _vp], _i32),
    "cpapr_run": ([_vp, _i32, ctypes.POINTER(alto_apr_params), _vp, _vp, _vp, _vp,
                   ctypes.POINTER(alto_apr_stats), _vp], _i32),
    "alto_autotune": ([_vp, _i32, _vp, _i32, _vp, _i32, _vp, ctypes.POINTER(alto_tune_result)], _i32),
    "alto_profile_enable": ([_vp, _i32], _i32),
    "alto_profile_read": ([_vp, ctypes.POINTER(alto_profile), _i32], _i32),
    "alto_kernel_launches": ([], _u64),
    "alto_last_error": ([], ctypes.c_char_p),
    "alto_version": ([], _i32),
}

_lib: Optional[ctypes.CDLL] = None


def alto_kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().alto_kernel_launches())


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib() -> ctypes.CDLL:
    """Load the in-tree libalto.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libalto.so not built ({LIB_PATH}); run "
                               "paper_2403_06348_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        msg = lib().alto_last_error()
        raise AltoError(status, msg.decode() if msg else "")


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


# ---------------------------------------------------------------------------
# C-named entry points (argument marshalling only)
# ---------------------------------------------------------------------------

def host_array(x, np_dtype, what: str = "array") -> np.ndarray:
    """A host array (numpy or CPU tensor) as a C-contiguous ``np_dtype`` array,
    without a copy where the bits already fit: int32 coordinates are read as
    uint32 in place, so a pinned buffer reaches the library as pinned memory
    (a negative coordinate then fails the library's range check). Wider or
    signed integer coordinates are converted only when every value fits
    uint32; otherwise ValueError (a silent wrap would encode another tensor)."""
    if not isinstance(x, np.ndarray):
        x = x.numpy()
    if np_dtype == np.uint32 and x.dtype == np.int32:
        x = x.view(np.uint32)
    if np_dtype == np.uint32 and x.dtype != np.uint32:
        if not np.issubdtype(x.dtype, np.integer):
            raise TypeError(f"{what}: host array of dtype {x.dtype}; expected integers")
        if x.size and (int(x.min()) < 0 or int(x.max()) > 0xFFFFFFFF):
            raise ValueError(f"{what}: values outside [0, 2^32) cannot be coordinates")
    return np.ascontiguousarray(x, dtype=np_dtype)


def alto_encode(coords, vals, dims: Sequence[int], stream=None, allocator=None) -> "AltoTensor":
    """Encode a COO tensor. ``coords`` is [nmodes, nnz] uint32/int32 and ``vals``
    [nnz] float32, each a CUDA tensor or a (host) numpy array / CPU tensor."""
    keep = []

    def prep(x, np_dtype, what):
        if isinstance(x, np.ndarray) or x.device.type == "cpu":
            a = host_array(x, np_dtype, what)
            keep.append(a)
            return a.ctypes.data
        # device memory goes to the library as a raw pointer, read as uint32
        # coordinates / float32 values: any other element type would be
        # misread (an int64 coordinate's high word as the next coordinate)
        torch = _torch()
        ok = (torch.int32, getattr(torch, "uint32", torch.int32)) if np_dtype == np.uint32 \
            else (torch.float32,)
        if x.dtype not in ok:
            raise TypeError(f"{what}: CUDA tensor of dtype {x.dtype}; expected "
                            f"{' or '.join(str(d) for d in ok)}")
        x = x.contiguous()
        keep.append(x)
        return x.data_ptr()

    nmodes = len(dims)
    if hasattr(coords, "shape") and coords.shape[0] != nmodes:
        raise ValueError("coords must be [nmodes, nnz]")
    nnz = int(coords.shape[1]) if nmodes else 0
    cp = prep(coords, np.uint32, "coords")
    vp = prep(vals, np.float32, "vals")
    dims_a = (ctypes.c_uint64 * nmodes)(*[int(d) for d in dims])
    h = ctypes.c_void_p()
    al = ctypes.byref(allocator) if allocator is not None else None
    _check(lib().alto_encode(cp, vp, dims_a, nmodes, nnz, al, _stream_ptr(stream), ctypes.byref(h)))
    return AltoTensor(h, tuple(int(d) for d in dims), nnz, allocator)


def _factor_dtype(factors, mode: int) -> int:
    """ALTO_BF16 when the input factors are bfloat16 tensors, else ALTO_F32."""
    for m, f in enumerate(factors):
        if m != mode and f is not None and getattr(f, "dtype", None) is not None \
                and str(f.dtype) == "torch.bfloat16":
            return ALTO_BF16
    return ALTO_F32


def alto_mttkrp(t: "AltoTensor", mode: int, factors, R: int, out, dtype: int = ALTO_F32,
                stream=None) -> None:
    arr = (ctypes.c_void_p * t.nmodes)(*[_ptr(f) for f in factors])
    _check(lib().alto_mttkrp(t.handle, int(mode), arr, int(dtype), int(R), _ptr(out),
                             _stream_ptr(stream)))


def alto_mttkrp_noalloc(t: "AltoTensor", mode: int, factors, R: int, out, dtype: Optional[int] = None,
                        stream=None) -> None:
    """Pull-variant MTTKRP that allocates nothing (scratch in the library's fixed
    device array); the mode's pull lists must exist (see include/alto.h).
    ``dtype`` defaults to the factors' element type (ALTO_BF16 for bfloat16)."""
    if dtype is None:
        dtype = _factor_dtype(factors, mode)
    arr = (ctypes.c_void_p * t.nmodes)(*[_ptr(f) for f in factors])
    _check(lib().alto_mttkrp_noalloc(t.handle, int(mode), arr, int(dtype), int(R), _ptr(out),
                                     _stream_ptr(stream)))


def cpals_run(t: "AltoTensor", R: int, iters: int, factors, lam, fits: Optional[np.ndarray] = None,
              tol: float = 0.0, stream=None) -> int:
    arr = (ctypes.c_void_p * t.nmodes)(*[_ptr(f) for f in factors])
    done = ctypes.c_int(0)
    _check(lib().cpals_run(t.handle, int(R), int(iters), arr, _ptr(lam),
                           _ptr(fits) if fits is not None else None, float(tol),
                           ctypes.byref(done), _stream_ptr(stream)))
    return int(done.value)


def alto_mttkrp_grouped(problems, dtype: int = ALTO_F32, stream=None) -> None:
    """One grouped launch over ``problems``: a sequence of
    (tensor, mode, factors, R, out) tuples (factors and out CUDA tensors)."""
    n = len(problems)
    if n == 0:
        return
    hs = (ctypes.c_void_p * n)(*[p[0].handle for p in problems])
    modes = (ctypes.c_int * n)(*[int(p[1]) for p in problems])
    fac_arrays = [(ctypes.c_void_p * p[0].nmodes)(*[_ptr(f) for f in p[2]]) for p in problems]
    facs = (ctypes.c_void_p * n)(*[ctypes.cast(a, ctypes.c_void_p).value for a in fac_arrays])
    Rs = (ctypes.c_int * n)(*[int(p[3]) for p in problems])
    outs = (ctypes.c_void_p * n)(*[_ptr(p[4]) for p in problems])
    _check(lib().alto_mttkrp_grouped(n, hs, modes, facs, Rs, int(dtype), outs,
                                     _stream_ptr(stream)))


def alto_fill_uniform(dst, seed: int, stream=None) -> None:
    """Seeded uniform [0, 1) fill of a float32 CUDA tensor (see include/alto.h)."""
    _check(lib().alto_fill_uniform(_ptr(dst), int(dst.numel()), int(seed), _stream_ptr(stream)))


def alto_cpals_footprint(dims: Sequence[int], nnz: int, R: int, iters: int) -> Tuple[int, int]:
    """(resident, peak) device bytes of one CP-ALS run in a batch."""
    d = (ctypes.c_uint64 * len(dims))(*[int(x) for x in dims])
    res, peak = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().alto_cpals_footprint(len(dims), d, int(nnz), int(R), int(iters),
                                      ctypes.byref(res), ctypes.byref(peak)))
    return int(res.value), int(peak.value)


class Batch:
    """CP-ALS batch (alto_batch_*): runs on many tensors advanced together,
    one mode update of every active run per step, replayed from a CUDA graph."""

    def __init__(self, max_slots: int = 1024, stream=None):
        torch = _torch()
        self._b = None
        # the batch runs on its own stream; inputs made on the caller's current
        # stream are ordered before each add, and results after each result()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        b = ctypes.c_void_p()
        _check(lib().alto_batch_create(int(max_slots), None, _stream_ptr(self.stream),
                                       ctypes.byref(b)))
        self._b = b
        self._tensors = {}

    def add(self, t: "AltoTensor", R: int, iters: int, factors, tol: float = 0.0) -> int:
        torch = _torch()
        self.stream.wait_stream(torch.cuda.current_stream())
        arr = (ctypes.c_void_p * t.nmodes)(*[_ptr(f) for f in factors])
        slot = ctypes.c_int(-1)
        _check(lib().alto_batch_add(self._b, t.handle, int(R), int(iters), float(tol), arr,
                                    ctypes.byref(slot)))
        self._tensors[slot.value] = t
        return int(slot.value)

    @staticmethod
    def prepare(t: "AltoTensor", R: int) -> None:
        """alto_batch_prepare: the handle's batch set-up, on its own stream."""
        _check(lib().alto_batch_prepare(t.handle, int(R)))

    def step(self, nsteps: int = 1) -> None:
        _check(lib().alto_batch_step(self._b, int(nsteps)))

    def poll(self, wait: bool = False, cap: int = 4096) -> List[int]:
        buf = (ctypes.c_int * cap)()
        n = ctypes.c_int(0)
        _check(lib().alto_batch_poll(self._b, 1 if wait else 0, buf, cap, ctypes.byref(n)))
        return [int(buf[i]) for i in range(n.value)]

    def result(self, slot: int, factors, lam=None, fits=None) -> Tuple[int, int]:
        """Enqueue the run's normalised factors (and lambda / fits) into the
        given buffers; returns (iters_done, run_status)."""
        t = self._tensors[slot]
        arr = (ctypes.c_void_p * t.nmodes)(*[_ptr(f) for f in factors])
        done, st = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().alto_batch_result(self._b, int(slot), arr, _ptr(lam) if lam is not None else None,
                                       _ptr(fits) if fits is not None else None, ctypes.byref(done),
                                       ctypes.byref(st)))
        _torch().cuda.current_stream().wait_stream(self.stream)
        return int(done.value), int(st.value)

    def copy_out(self, slot: int, factors, lam=None, fits=None, stream=None) -> None:
        """alto_batch_copy_out: the slot's results (after result()) into the
        given buffers; may run on another thread until remove()."""
        t = self._tensors[slot]
        arr = (ctypes.c_void_p * t.nmodes)(*[_ptr(f) for f in factors])
        _check(lib().alto_batch_copy_out(self._b, int(slot), arr, _ptr(lam) if lam is not None else None,
                                         _ptr(fits) if fits is not None else None,
                                         _stream_ptr(stream)))

    def remove(self, slot: int) -> None:
        _check(lib().alto_batch_remove(self._b, int(slot)))
        self._tensors.pop(slot, None)

    def sync(self) -> None:
        _check(lib().alto_batch_sync(self._b))

    def info(self) -> alto_batch_info:
        i = alto_batch_info()
        _check(lib().alto_batch_query(self._b, ctypes.byref(i)))
        return i

    def free(self) -> None:
        if self._b:
            lib().alto_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# handle wrapper
# ---------------------------------------------------------------------------

class AltoTensor:
    """An encoded tensor on the current CUDA device."""

    def __init__(self, handle: ctypes.c_void_p, dims: Tuple[int, ...], nnz: int, allocator=None):
        self.handle = handle
        self.dims = dims
        self.nnz = nnz
        self._allocator = allocator  # keep the callbacks alive

    @property
    def nmodes(self) -> int:
        return len(self.dims)

    def free(self) -> None:
        if self.handle:
            lib().alto_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def query(self) -> alto_info:
        info = alto_info()
        _check(lib().alto_query(self.handle, ctypes.byref(info)))
        return info

    def profile_enable(self, on: bool = True) -> None:
        _check(lib().alto_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, reset: bool = False) -> dict:
        p = alto_profile()
        _check(lib().alto_profile_read(self.handle, ctypes.byref(p), 1 if reset else 0))
        return {k: (int(p.launches[i]), float(p.ms[i])) for i, k in enumerate(PROF_KINDS)}

    def set_partitions(self, nparts: int, stream=None) -> None:
        _check(lib().alto_set_partitions(self.handle, int(nparts), _stream_ptr(stream)))

    def partition(self) -> Tuple[np.ndarray, np.ndarray]:
        info = self.query()
        L = int(info.nparts)
        starts = np.empty(L + 1, dtype=np.uint64)
        iv = np.empty((L, self.nmodes, 2), dtype=np.uint32)
        _check(lib().alto_copy_partition(self.handle, starts.ctypes.data, iv.ctypes.data))
        return starts, iv

    def encoded(self, stream=None):
        torch = _torch()
        info = self.query()
        kw = int(info.key_words)
        keys = torch.empty((self.nnz, kw), dtype=torch.int64, device="cuda")
        vals = torch.empty(self.nnz, dtype=torch.float32, device="cuda")
        _check(lib().alto_copy_encoded(self.handle, _ptr(keys), _ptr(vals), _stream_ptr(stream)))
        return keys, vals

    def decode(self, stream=None):
        torch = _torch()
        coords = torch.empty((self.nmodes, self.nnz), dtype=torch.int32, device="cuda")
        vals = torch.empty(self.nnz, dtype=torch.float32, device="cuda")
        _check(lib().alto_decode(self.handle, _ptr(coords), _ptr(vals), _stream_ptr(stream)))
        return coords, vals

    def hot_rows(self, mode: int) -> np.ndarray:
        buf = np.empty(ALTO_MAX_HOT, dtype=np.uint32)
        cnt = ctypes.c_uint32(0)
        _check(lib().alto_copy_hot_rows(self.handle, int(mode), buf.ctypes.data, ALTO_MAX_HOT,
                                        ctypes.byref(cnt)))
        return buf[: cnt.value].copy()

    def set_mode_plan(self, mode: int, variant: int = VARIANT_AUTO, cols_per_lane: int = 0,
                      hot_rows: int = -1) -> None:
        p = alto_mode_plan(int(variant), int(cols_per_lane), int(hot_rows))
        _check(lib().alto_set_mode_plan(self.handle, int(mode), ctypes.byref(p)))

    def get_mode_plan(self, mode: int, R: int) -> Tuple[int, int, int]:
        p = alto_mode_plan()
        _check(lib().alto_get_mode_plan(self.handle, int(mode), int(R), ctypes.byref(p)))
        return int(p.variant), int(p.cols_per_lane), int(p.hot_rows)

    def mttkrp(self, mode: int, factors, R: Optional[int] = None, out=None, dtype=None,
               stream=None):
        torch = _torch()
        R = int(R if R is not None else factors[(mode + 1) % self.nmodes].shape[1])
        code = dtype if dtype is not None else _factor_dtype(factors, mode)
        if out is None:
            rows = self.dims[mode] if 0 <= mode < self.nmodes else 1  # the C call rejects bad modes
            out = torch.empty((rows, R), dtype=torch.float32, device="cuda")
        alto_mttkrp(self, mode, factors, R, out, code, stream)
        return out

    def build_pos_out(self, mode: int = -1, nparts: int = 0, stream=None) -> None:
        """alto_build_pos_out: the stored output-oriented order of one mode (-1: all)."""
        _check(lib().alto_build_pos_out(self.handle, int(mode), int(nparts), _stream_ptr(stream)))

    def pos_out(self, mode: int, stream=None) -> Tuple[np.ndarray, int]:
        """alto_copy_pos_out: (the stored order of `mode` as uint32 positions, its segment count)."""
        buf = np.empty(max(self.nnz, 1), dtype=np.uint32)
        L = ctypes.c_uint64(0)
        _check(lib().alto_copy_pos_out(self.handle, int(mode), buf.ctypes.data, ctypes.byref(L),
                                       _stream_ptr(stream)))
        return buf[: self.nnz], int(L.value)

    def free_pos_out(self, mode: int = -1) -> None:
        _check(lib().alto_free_pos_out(self.handle, int(mode)))

    def autotune(self, factors, R: int, out=None, segments: bool = True, dtype=None,
                 stream=None, output: bool = False) -> dict:
        """alto_autotune: measured per-mode plan (and segment count); the
        winners stay set on the handle. ``output`` adds the OUTPUT plan (the
        stored order) to the candidates. Returns the report as a dict."""
        torch = _torch()
        code = ALTO_F32
        if dtype is not None:
            code = dtype
        elif any(f is not None and f.dtype == torch.bfloat16 for f in factors):
            code = ALTO_BF16
        if out is None:
            out = torch.empty((max(self.dims), R), dtype=torch.float32, device="cuda")
        arr = (ctypes.c_void_p * self.nmodes)(*[_ptr(f) for f in factors])
        res = alto_tune_result()
        _check(lib().alto_autotune(self.handle, int(R), arr, int(code), _ptr(out),
                                   (ALTO_TUNE_SEGMENTS if segments else 0)
                                   | (ALTO_TUNE_OUTPUT if output else 0), _stream_ptr(stream),
                                   ctypes.byref(res)))
        n = self.nmodes
        return {"plans": [(int(res.plan[i].variant), int(res.plan[i].cols_per_lane),
                           int(res.plan[i].hot_rows)) for i in range(n)],
                "ms": [float(res.ms[i]) for i in range(n)],
                "default_ms": [float(res.default_ms[i]) for i in range(n)],
                "nparts": int(res.nparts), "candidates": int(res.candidates)}

    def phi(self, mode: int, factors, B, R: int, eps: float = 1e-10, pre: bool = False, out=None,
            stream=None):
        """alto_phi: the CP-APR model update Phi of Alg. 5 for one mode."""
        torch = _torch()
        if out is None:
            out = torch.empty((self.dims[mode], R), dtype=torch.float32, device="cuda")
        arr = (ctypes.c_void_p * self.nmodes)(*[_ptr(f) for f in factors])
        _check(lib().alto_phi(self.handle, int(mode), arr, _ptr(B), int(R), float(eps),
                              1 if pre else 0, _ptr(out), _stream_ptr(stream)))
        return out

    def cpapr(self, R: int, factors, k_max: int, l_max: int = 10, tau: float = 1e-4,
              kappa: float = 1e-2, kappa_tol: float = 1e-10, eps: float = 1e-10,
              variant: int = APR_AUTO, stream=None) -> dict:
        """cpapr_run in place on ``factors`` (CUDA float32 tensors or numpy
        float32 arrays). Returns lambda, objectives, inner steps and stats."""
        torch = _torch()
        on_dev = not isinstance(factors[0], np.ndarray)
        lam = torch.empty(R, dtype=torch.float64, device="cuda") if on_dev else np.empty(R)
        obj = np.zeros(k_max)
        steps = np.zeros((k_max, self.nmodes), dtype=np.int32)
        prm = alto_apr_params(int(k_max), int(l_max), float(tau), float(kappa), float(kappa_tol),
                              float(eps), int(variant))
        st = alto_apr_stats()
        arr = (ctypes.c_void_p * self.nmodes)(*[_ptr(f) for f in factors])
        _check(lib().cpapr_run(self.handle, int(R), ctypes.byref(prm), arr, _ptr(lam), obj.ctypes.data,
                               steps.ctypes.data, ctypes.byref(st), _stream_ptr(stream)))
        k = int(st.outer_done)
        return {"lam": lam.cpu().numpy() if on_dev else lam, "objective": obj[:k].tolist(),
                "inner": steps[:k].tolist(), "outer_done": k, "converged": bool(st.converged),
                "inner_steps_total": int(st.inner_steps_total), "pre_modes": int(st.pre_modes)}

    def cpals(self, R: int, iters: int, factors, tol: float = 0.0, stream=None):
        """Run CP-ALS in place on ``factors`` (CUDA float32 tensors or numpy
        float32 arrays). Returns (lambda float64 numpy [R], fits list)."""
        torch = _torch()
        on_dev = not isinstance(factors[0], np.ndarray)
        lam = torch.empty(R, dtype=torch.float64, device="cuda") if on_dev else np.empty(R)
        fits = np.zeros(iters, dtype=np.float64)
        done = cpals_run(self, R, iters, factors, lam, fits, tol, stream)
        lam_np = lam.cpu().numpy() if on_dev else lam
        return lam_np, fits[:done].tolist()
