"""Helpers shared by the GPU parity tests (inputs, conversions, comparisons)."""
import numpy as np

import paper_2403_06348_gb300 as alto

_built = False


def ensure_built():
    global _built
    if not _built:
        alto.build()
        _built = True


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def coords_dev(coords):
    import torch
    return to_dev(coords.astype(np.uint32).view(np.int32), torch.int32)


def encode(coords, vals, dims):
    return alto.alto_encode(coords_dev(coords), to_dev(vals.astype(np.float32)), dims)


def rand_tensor(dims, M, seed, dist="uniform"):
    rng = np.random.default_rng(seed)
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    vals = (1.0 - rng.random(M)).astype(np.float32)
    return coords, vals


def rand_factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.random((d, R), dtype=np.float32) for d in dims]


def gpu_factors(factors, dtype=None):
    import torch
    return [to_dev(f, dtype if dtype is not None else torch.float32) for f in factors]
