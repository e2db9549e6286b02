"""ctypes wrapper and build step for the plain C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

from . import alto_ref

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coo_ref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    """Compile coo_ref.c with gcc -O2 -fopenmp into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        _lib.oracle_mttkrp_f64.argtypes = [i32, u64, vp, vp, vp, vp, i32, i32, vp, i32]
        _lib.oracle_mttkrp_f64.restype = i32
        _lib.oracle_mttkrp_rows_f64.argtypes = [i32, u64, vp, vp, vp, vp, i32, i32, vp,
                                                ctypes.c_int64, vp]
        _lib.oracle_mttkrp_rows_f64.restype = i32
        _lib.oracle_linearize.argtypes = [i32, u64, vp, vp, vp, i32, vp]
        _lib.oracle_linearize.restype = None
        _lib.oracle_max_threads.restype = i32
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _prep(coords, vals, dims, factors):
    coords = np.ascontiguousarray(coords, dtype=np.uint32)
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    dims_a = np.ascontiguousarray(np.asarray(dims, dtype=np.uint64))
    fs = [np.ascontiguousarray(f, dtype=np.float32) for f in factors]
    ptrs = (ctypes.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    return coords, vals, dims_a, fs, ptrs


def mttkrp(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int],
           factors: Sequence[np.ndarray], mode: int, nthreads: int = 1) -> np.ndarray:
    """fp64 MTTKRP of one mode by its definition (float32 inputs)."""
    coords, vals, dims_a, fs, ptrs = _prep(coords, vals, dims, factors)
    R = fs[0].shape[1]
    out = np.empty((int(dims[mode]), R), dtype=np.float64)
    rc = lib().oracle_mttkrp_f64(len(dims), coords.shape[1], coords.ctypes.data,
                                 vals.ctypes.data, dims_a.ctypes.data, ptrs, R, mode,
                                 out.ctypes.data, int(nthreads))
    if rc != 0:
        raise MemoryError("oracle_mttkrp_f64 allocation failed")
    return out


def mttkrp_rows(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int],
                factors: Sequence[np.ndarray], mode: int, rows: np.ndarray) -> np.ndarray:
    """fp64 MTTKRP restricted to the listed (distinct) output rows."""
    coords, vals, dims_a, fs, ptrs = _prep(coords, vals, dims, factors)
    R = fs[0].shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    out = np.empty((rows.shape[0], R), dtype=np.float64)
    rc = lib().oracle_mttkrp_rows_f64(len(dims), coords.shape[1], coords.ctypes.data,
                                      vals.ctypes.data, dims_a.ctypes.data, ptrs, R, mode,
                                      rows.ctypes.data, rows.shape[0], out.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_mttkrp_rows_f64 allocation failed")
    return out


def linearize(coords: np.ndarray, dims: Sequence[int]) -> np.ndarray:
    """Keys as uint64 [M, kw] (kw words, low word first), by the bit plan of alto_ref."""
    plan = alto_ref.bit_plan(dims)
    kw = alto_ref.key_width_words(plan.nbits)
    coords = np.ascontiguousarray(coords, dtype=np.uint32)
    M = coords.shape[1]
    bits = np.asarray(plan.bits, dtype=np.int32)
    pos = np.zeros((len(dims), 32), dtype=np.int32)
    for n in range(len(dims)):
        pos[n, :plan.bits[n]] = plan.positions[n]
    keys = np.empty((M, kw), dtype=np.uint64)
    lib().oracle_linearize(len(dims), M, coords.ctypes.data, bits.ctypes.data,
                           pos.ctypes.data, kw, keys.ctypes.data)
    return keys
