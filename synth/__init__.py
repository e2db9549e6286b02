"""Seeded synthetic sparse tensors shaped like the paper's workloads.

This module only draws random inputs. It holds none of the method's
arithmetic (no linearization, ordering, partitioning or MTTKRP), so both the
CUDA path and the CPU oracle can consume its arrays without sharing code.

Every generator is a pure function of its arguments and a seed (numpy PCG64).
Coordinates are 0-based uint32 arrays laid out structure-of-arrays
``coords[nmodes, nnz]``; values are float32 ``vals[nnz]``.

Distributions:

* ``uniform``  -- ``Generator.integers(0, I)``.
* ``zipf s``   -- bounded Zipf on {0..I-1}, p(k) proportional to (k+1)^-s,
  drawn by exact inverse CDF (fp64 cumulative sum plus a guide table, then a
  short forward scan), followed by a seeded permutation of the rank -> index
  map so that hot rows are scattered over the mode as in real data.
* values: ``uniform01`` = U(0,1] (1 - U[0,1)), ``lognormal`` = lognormal(0,1),
  ``poisson3p1`` = Poisson(3) + 1.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20240311


@dataclasses.dataclass(frozen=True)
class TensorSpec:
    """Shape, nonzero count and distributions of one synthetic tensor."""

    name: str
    dims: Tuple[int, ...]
    nnz: int
    coord_dist: Tuple[str, ...]          # per mode: "uniform" or "zipf:<s>"
    value_dist: str                      # "uniform01" | "lognormal" | "poisson3p1"
    rank: int
    distinct: bool = False               # redraw duplicate coordinates
    seed: int = BASE_SEED
    permute_hot: bool = True             # scatter Zipf ranks by a permutation


# The four single-tensor workloads, named below by what they are: a small
# uniform 3-mode tensor the oracle finishes in seconds, the 1e8-nonzero Zipf
# 3-mode tensor of the headline measurement, a 2e8-nonzero 4-mode count
# tensor, and a 1.5e8-nonzero 5-mode Zipf tensor with 128-bit positions.
CONFIGS: List[TensorSpec] = [
    TensorSpec("uniform3d_1000x800x600_1e5_r16", (1000, 800, 600), 100_000,
               ("uniform",) * 3, "uniform01", 16, distinct=True, seed=BASE_SEED + 0),
    TensorSpec("zipf3d_10Mx2Mx50k_1e8_r32", (10_000_000, 2_000_000, 50_000), 100_000_000,
               ("zipf:1.1",) * 3, "lognormal", 32, seed=BASE_SEED + 1),
    TensorSpec("count4d_1Mx500kx200x24_2e8_r16", (1_000_000, 500_000, 200, 24), 200_000_000,
               ("zipf:1.2", "zipf:1.2", "uniform", "uniform"), "poisson3p1", 16,
               seed=BASE_SEED + 2),
    TensorSpec("zipf5d_2Mx100kx10kx1000x50_1.5e8_r64", (2_000_000, 100_000, 10_000, 1000, 50),
               150_000_000, ("zipf:1.1",) * 5, "uniform01", 64, seed=BASE_SEED + 3),
]

UNIFORM3D, ZIPF3D, COUNT4D, ZIPF5D = CONFIGS


def scaled(spec: TensorSpec, nnz: int, dims: Optional[Sequence[int]] = None,
           name: Optional[str] = None) -> TensorSpec:
    """Same distributions with another nonzero count (and optionally dims)."""
    return dataclasses.replace(spec, nnz=int(nnz), dims=tuple(dims) if dims else spec.dims,
                               name=name or f"{spec.name}@{nnz}")


# ---------------------------------------------------------------------------
# samplers
# ---------------------------------------------------------------------------

def _zipf_cdf(size: int, s: float) -> np.ndarray:
    k = np.arange(1, size + 1, dtype=np.float64)
    w = k ** (-s)
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def bounded_zipf(rng: np.random.Generator, size: int, s: float, count: int,
                 chunk: int = 1 << 23) -> np.ndarray:
    """Exact inverse-CDF draws of ranks in [0, size) with p(k) ~ (k+1)^-s.

    For a uniform u the drawn rank is the smallest k with cdf[k] > u. A guide
    table ``g[j] = #{k : cdf[k] <= j/G}`` gives a starting rank that is never
    past the answer; a short vectorised forward scan finishes the search.
    """
    cdf = _zipf_cdf(size, s)
    G = size
    guide = np.searchsorted(cdf, np.arange(G, dtype=np.float64) / G, side="right")
    out = np.empty(count, dtype=np.int64)
    for lo in range(0, count, chunk):
        hi = min(count, lo + chunk)
        u = rng.random(hi - lo)
        k = guide[np.minimum((u * G).astype(np.int64), G - 1)]
        active = np.nonzero(cdf[k] <= u)[0]
        while active.size:
            k[active] += 1
            still = cdf[k[active]] <= u[active]
            active = active[still]
        out[lo:hi] = k
    return out


def _draw_mode(rng: np.random.Generator, dist: str, size: int, count: int,
               permute: bool) -> np.ndarray:
    if dist == "uniform":
        return rng.integers(0, size, count, dtype=np.int64)
    if dist.startswith("zipf:"):
        s = float(dist.split(":", 1)[1])
        ranks = bounded_zipf(rng, size, s, count)
        if permute:
            perm = rng.permutation(size)
            return perm[ranks]
        return ranks
    raise ValueError(f"unknown coordinate distribution {dist!r}")


def _draw_values(rng: np.random.Generator, dist: str, count: int) -> np.ndarray:
    if dist == "uniform01":
        v = 1.0 - rng.random(count)
    elif dist == "lognormal":
        v = rng.lognormal(0.0, 1.0, count)
    elif dist == "poisson3p1":
        v = rng.poisson(3.0, count) + 1.0
    else:
        raise ValueError(f"unknown value distribution {dist!r}")
    return v.astype(np.float32)


def generate(spec: TensorSpec) -> Tuple[np.ndarray, np.ndarray]:
    """Return ``(coords uint32 [N, nnz], vals float32 [nnz])`` for ``spec``."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    N = len(spec.dims)
    M = spec.nnz
    coords = np.empty((N, M), dtype=np.uint32)
    for n in range(N):
        coords[n] = _draw_mode(rng, spec.coord_dist[n], spec.dims[n], M, spec.permute_hot)
    if spec.distinct and M > 0:
        coords = _redraw_duplicates(rng, spec, coords)
    vals = _draw_values(rng, spec.value_dist, M)
    return coords, vals


def _redraw_duplicates(rng: np.random.Generator, spec: TensorSpec,
                       coords: np.ndarray) -> np.ndarray:
    """Redraw later copies of repeated coordinate tuples until all are distinct."""
    dims = np.asarray(spec.dims, dtype=np.int64)
    total = int(np.prod([float(d) for d in dims]))
    if spec.nnz > total:
        raise ValueError("more distinct nonzeros requested than cells")
    for _ in range(1000):
        flat = np.ravel_multi_index(tuple(coords.astype(np.int64)), tuple(spec.dims))
        _, first = np.unique(flat, return_index=True)
        dup = np.ones(flat.shape[0], dtype=bool)
        dup[first] = False
        idx = np.nonzero(dup)[0]
        if idx.size == 0:
            return coords
        for n in range(len(spec.dims)):
            coords[n, idx] = _draw_mode(rng, spec.coord_dist[n], spec.dims[n], idx.size,
                                        spec.permute_hot)
    raise RuntimeError("could not make coordinates distinct")


def factors(dims: Sequence[int], rank: int, seed: int) -> List[np.ndarray]:
    """Seeded factor matrices, float32 U[0,1), row-major ``[I_n, rank]``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.random((int(I), rank), dtype=np.float32) for I in dims]


# ---------------------------------------------------------------------------
# on-disk cache for the large configurations
# ---------------------------------------------------------------------------

def cache_dir() -> str:
    d = os.environ.get("ALTO_SYNTH_CACHE", os.path.join("/tmp", "alto_synth_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def cached(spec: TensorSpec) -> Tuple[np.ndarray, np.ndarray]:
    """``generate(spec)`` memoised as .npy files (memory-mapped on reload)."""
    key = f"{spec.name}_{spec.nnz}_{spec.seed}_{'x'.join(map(str, spec.dims))}"
    key = key.replace(":", "_").replace("@", "_")
    d = cache_dir()
    pc, pv = os.path.join(d, key + "_coords.npy"), os.path.join(d, key + "_vals.npy")
    if os.path.exists(pc) and os.path.exists(pv):
        return np.load(pc, mmap_mode="r"), np.load(pv, mmap_mode="r")
    coords, vals = generate(spec)
    tmpc, tmpv = pc + ".tmp.npy", pv + ".tmp.npy"
    np.save(tmpc, coords)
    np.save(tmpv, vals)
    os.replace(tmpc, pc)
    os.replace(tmpv, pv)
    return coords, vals


# ---------------------------------------------------------------------------
# serving workload: a stream of CP-ALS requests
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    dims: Tuple[int, ...]
    nnz: int
    rank: int
    iters: int
    seed: int


def request_stream(count: int = 2000, rate_per_s: float = 200.0, seed: int = BASE_SEED + 4,
                   dim_range=(100, 1_000_000), nnz_range=(1_000, 10_000_000),
                   modes=(3, 4, 5), ranks=(8, 16, 32), iters: int = 20) -> List[Request]:
    """Poisson arrivals of CP-ALS requests with log-uniform dims and nnz."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, count)
    t = np.cumsum(gaps)
    out = []
    for i in range(count):
        N = int(rng.choice(modes))
        dims = tuple(int(round(math.exp(rng.uniform(math.log(dim_range[0]),
                                                    math.log(dim_range[1])))))
                     for _ in range(N))
        nnz = int(round(math.exp(rng.uniform(math.log(nnz_range[0]), math.log(nnz_range[1])))))
        out.append(Request(i, float(t[i]), dims, nnz, int(rng.choice(ranks)), iters,
                           int(rng.integers(0, 2**31 - 1))))
    return out


def request_tensor(req: Request) -> Tuple[np.ndarray, np.ndarray]:
    spec = TensorSpec(f"req{req.rid}", req.dims, req.nnz, ("zipf:1.1",) * len(req.dims),
                      "uniform01", req.rank, seed=req.seed)
    return generate(spec)


def request_pool_stream(count: int = 2000, pool: int = 64, rate_per_s: float = 200.0,
                        seed: int = BASE_SEED + 4, dim_range=(100, 1_000_000),
                        nnz_range=(1_000, 10_000_000), modes=(3, 4, 5), ranks=(8, 16, 32),
                        iters: int = 20) -> Tuple[List[Request], List[Request]]:
    """The serving workload with a bounded amount of tensor data to generate.

    ``pool`` distinct tensors are drawn with their nonzero counts at the
    midpoints of ``pool`` equal log-spaced bins of ``nnz_range`` (so the pool
    follows the log-uniform law, mean included) and dims, order and rank drawn
    as in ``request_stream``. The ``count`` requests arrive as a Poisson
    stream at ``rate_per_s``; request i uses pool entry perm[i mod pool] of a
    seeded permutation, with its own rank and initial-factor seed. Returns
    (pool, requests); a request's ``rid`` is its pool index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = math.log(nnz_range[0]), math.log(nnz_range[1])
    entries = []
    for j in range(pool):
        N = int(rng.choice(modes))
        dims = tuple(int(round(math.exp(rng.uniform(math.log(dim_range[0]),
                                                    math.log(dim_range[1])))))
                     for _ in range(N))
        nnz = int(round(math.exp(lo + (j + 0.5) / pool * (hi - lo))))
        entries.append(Request(j, 0.0, dims, nnz, int(rng.choice(ranks)), iters,
                               int(rng.integers(0, 2**31 - 1))))
    perm = rng.permutation(pool)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, count))
    reqs = []
    for i in range(count):
        e = entries[int(perm[i % pool])]
        reqs.append(Request(e.rid, float(t[i]), e.dims, e.nnz, int(rng.choice(ranks)), iters,
                            int(rng.integers(0, 2**31 - 1))))
    return entries, reqs
