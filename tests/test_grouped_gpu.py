"""Grouped MTTKRP (alto_mttkrp_grouped): many tensors of different order, key
width and rank in one launch, each output against the fp64 oracle with the
single-tensor bar (fp32 <= 1e-5 row-relative, bf16 <= 1e-2, empty rows exactly 0).
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from oracle import cref
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _zipf_tensor(dims, nnz, seed):
    spec = synth.TensorSpec(f"g{seed}", tuple(dims), nnz, ("zipf:1.1",) * len(dims), "uniform01", 8,
                            seed=seed)
    return synth.generate(spec)


# (dims, nnz, R): 3 to 6 modes, 64-bit and 128-bit positions, modes that stage
# their rows in shared memory (short) and modes that do not (long)
CASES = [
    ((300, 200, 100), 30_000, 16),
    ((50_000, 2_000, 300), 80_000, 32),
    ((40, 30, 20, 10), 20_000, 8),
    ((5_000, 300, 200, 50, 20), 50_000, 64),           # 5 modes
    ((2_000_000, 100_000, 10_000, 1000, 50), 60_000, 16),  # 68 bits: 128-bit positions
    ((30, 20, 16, 12, 10, 8), 15_000, 4),                # 6 modes: run-time decode
    ((100, 80, 60), 7, 16),                              # fewer nonzeros than a warp
]


def _problems(bf16=False, modes_of=None):
    import torch
    probs, refs = [], []
    for i, (dims, nnz, R) in enumerate(CASES):
        coords, vals = _zipf_tensor(dims, nnz, 100 + i)
        t = gu.encode(coords, vals, dims)
        A = gu.rand_factors(dims, R, 200 + i)
        Ad = gu.gpu_factors(A, torch.bfloat16 if bf16 else torch.float32)
        modes = modes_of(i, len(dims)) if modes_of else [i % len(dims)]
        for n in modes:
            out = torch.full((dims[n], R), 3.0, device="cuda")
            probs.append((t, n, Ad, R, out))
            refs.append(cref.mttkrp(coords, vals, dims, A, n, nthreads=4))
    return probs, refs


def _check(probs, refs, tol):
    for (t, n, _, R, out), ref in zip(probs, refs):
        got = out.cpu().numpy()
        err, bad_zero = ar.row_relative_error(got, ref)
        assert bad_zero == 0, f"dims {t.dims} mode {n}: rows without nonzeros are not 0"
        assert err <= tol, f"dims {t.dims} mode {n} R {R}: {err:.3g} > {tol}"


def test_grouped_mixed_orders_ranks_and_widths():
    import paper_2403_06348_gb300 as alto
    probs, refs = _problems()
    alto.alto_mttkrp_grouped(probs)
    _check(probs, refs, TOL_F32)


def test_grouped_every_mode_of_every_tensor():
    """The same handle several times in one launch, once per output mode."""
    import paper_2403_06348_gb300 as alto
    probs, refs = _problems(modes_of=lambda i, N: list(range(N)))
    alto.alto_mttkrp_grouped(probs)
    _check(probs, refs, TOL_F32)


def _bf16_bound(N):
    """Row-relative bound of bf16 factors against the fp32-factor oracle: each
    of the N-1 gathered values is rounded to 8 significant bits (relative
    error <= 2^-8), so a row made of one nonzero can be off by (N-1) 2^-8 plus
    the fp32 bar; 1e-2 holds as stated for N <= 3."""
    return max(TOL_BF16, (1 + 2.0 ** -8) ** (N - 1) - 1 + TOL_F32)


def test_grouped_bf16_factors():
    """Against the oracle on the bf16-rounded factors the kernel meets the fp32
    bar; against the oracle on the original factors the error is the bf16
    rounding, within its bound."""
    import torch
    import paper_2403_06348_gb300 as alto
    probs, refs = _problems(bf16=True, modes_of=lambda i, N: [0, N - 1])
    alto.alto_mttkrp_grouped(probs, dtype=alto.ALTO_BF16)
    for (t, n, Ad, R, out), ref in zip(probs, refs):
        got = out.cpu().numpy()
        err, bad_zero = ar.row_relative_error(got, ref)
        assert bad_zero == 0
        assert err <= _bf16_bound(t.nmodes), f"dims {t.dims} mode {n}: {err:.3g}"
        rounded = [a.float().cpu().numpy() for a in Ad]   # the bf16 values, exactly
        coords, vals = _zipf_tensor(t.dims, t.nnz, 100 + [c[0] for c in CASES].index(t.dims))
        ref_q = cref.mttkrp(coords, vals, t.dims, rounded, n, nthreads=4)
        err_q, _ = ar.row_relative_error(got, ref_q)
        assert err_q <= TOL_F32, f"dims {t.dims} mode {n}: kernel error {err_q:.3g}"


def test_grouped_equals_single_calls():
    import torch
    import paper_2403_06348_gb300 as alto
    probs, _ = _problems(modes_of=lambda i, N: [N // 2])
    alto.alto_mttkrp_grouped(probs)
    for t, n, Ad, R, out in probs:
        single = t.mttkrp(n, Ad, R)
        err, bad_zero = ar.row_relative_error(out.cpu().numpy(), single.double().cpu().numpy())
        assert bad_zero == 0 and err <= 2 * TOL_F32


def test_grouped_fine_and_coarse_segments():
    """Balance is by segment: tensors re-partitioned to very different segment
    sizes still give the same results."""
    import paper_2403_06348_gb300 as alto
    probs, refs = _problems(modes_of=lambda i, N: [0])
    for j, (t, *_rest) in enumerate(probs):
        t.set_partitions(1 if j % 2 else max(1, t.nnz // 64))
    alto.alto_mttkrp_grouped(probs)
    _check(probs, refs, TOL_F32)


def test_grouped_empty_and_bad_arguments():
    import torch
    import paper_2403_06348_gb300 as alto
    alto.alto_mttkrp_grouped([])
    coords, vals = gu.rand_tensor((10, 10, 10), 100, 1)
    t = gu.encode(coords, vals, (10, 10, 10))
    A = [torch.rand((10, 8), device="cuda") for _ in range(3)]
    out = torch.empty((10, 8), device="cuda")
    with pytest.raises(alto.AltoError) as e:
        alto.alto_mttkrp_grouped([(t, 0, A, 8, out), (t, 3, A, 8, out)])
    assert e.value.status == -1 and "problem 1" in str(e.value)
    with pytest.raises(alto.AltoError) as e:
        alto.alto_mttkrp_grouped([(t, 0, A, 12, out)])
    assert e.value.status == -4
