"""MTTKRP with the in-tile output-oriented traversal (TILED, TILED_LINE)
against the fp64 oracle, through the C ABI.

The kernel regroups every tile of 1024 consecutive nonzeros of the one ALTO
copy by output row, so the cases cover tile edges (fewer nonzeros than a
tile, exact multiples, one past), the three destinations of a run (rows
staged in shared memory, warm rows summed in replicas, all other rows), repeated
calls (the replicas must be left zero), 3- to 6-mode tensors, 64- and
128-bit positions, R from 4 to 64 with 4 or 8 columns per lane, and bf16
factors. Bar as every MTTKRP test: 1e-5 row-relative (fp32 factors), 1e-2
against the oracle on the original fp32 factors (bf16 factors).
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
TILED, TILED_LINE = 4, 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _check(t, coords, vals, dims, A, R, variant, cpl, bf16=False, modes=None, calls=1):
    import torch
    Ad = gu.gpu_factors(A, torch.bfloat16 if bf16 else torch.float32)
    for n in (modes if modes is not None else range(len(dims))):
        t.set_mode_plan(n, variant, cpl)
        ref = cref.mttkrp(coords, vals, dims, A, n, nthreads=4)
        for call in range(calls):
            out = torch.full((dims[n], R), float("nan"), device="cuda")
            t.mttkrp(n, Ad, R, out=out)
            got = out.cpu().numpy()
            err, bad_zero = ar.row_relative_error(got, ref)
            assert bad_zero == 0, f"mode {n} call {call}: rows without nonzeros are not exactly 0"
            lim = TOL_BF16 if bf16 else TOL_F32
            assert err <= lim, f"mode {n} call {call}: row-relative error {err:.3g} > {lim}"
        plan = t.get_mode_plan(n, R)
        assert plan[0] == variant, plan


@pytest.mark.parametrize("variant", [TILED, TILED_LINE])
@pytest.mark.parametrize("nnz", [1, 37, 1023, 1024, 1025, 4096, 5000, 70_001])
def test_tile_edges(variant, nnz):
    dims = (90, 70, 50)
    coords, vals = gu.rand_tensor(dims, nnz, nnz)
    t = gu.encode(coords, vals, dims)
    A = gu.rand_factors(dims, 16, 3)
    _check(t, coords, vals, dims, A, 16, variant, 8)
    _check(t, coords, vals, dims, A, 16, variant, 4)


@pytest.mark.parametrize("variant", [TILED, TILED_LINE])
@pytest.mark.parametrize("R", [4, 8, 16, 32, 64])
def test_ranks_and_lane_widths(variant, R):
    coords, vals = gu.rand_tensor((300, 200, 150), 60_000, R)
    dims = (300, 200, 150)
    t = gu.encode(coords, vals, dims)
    A = gu.rand_factors(dims, R, R)
    for cpl in (4, 8):
        _check(t, coords, vals, dims, A, R, variant, cpl)


@pytest.mark.parametrize("variant", [TILED, TILED_LINE])
def test_zipf_staged_and_warm_rows_two_calls(variant):
    """Skewed modes put hot rows in all three places (shared memory, warm
    replicas, the output); a second call must find the replicas zero."""
    spec = synth.scaled(synth.ZIPF3D, 2_000_000, dims=(3000, 2000, 1500))
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    for R in (32, 64):
        A = gu.rand_factors(spec.dims, R, 5)
        _check(t, coords, vals, spec.dims, A, R, variant, 8, calls=2)
        if R == 64:
            staged = t.get_mode_plan(0, R)[2]
            nhot = int(t.query().nhot[0])
            assert 0 < staged < min(nhot, 1024), (staged, nhot)   # warm rows exist


def test_zipf_full_mode_lengths_hot_rows():
    spec = synth.scaled(synth.ZIPF3D, 2_000_000)
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.rand_factors(spec.dims, 32, 6)
    for variant in (TILED, TILED_LINE):
        _check(t, coords, vals, spec.dims, A, 32, variant, 8)


@pytest.mark.parametrize("variant", [TILED, TILED_LINE])
def test_bf16_factors(variant):
    spec = synth.UNIFORM3D
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.rand_factors(spec.dims, 16, 2)
    for cpl in (4, 8):
        _check(t, coords, vals, spec.dims, A, 16, variant, cpl, bf16=True)


def test_five_modes_two_word_positions():
    spec = synth.scaled(synth.ZIPF5D, 300_000)
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    assert int(t.query().key_words) == 2
    A = gu.rand_factors(spec.dims, 64, 4)
    for variant in (TILED, TILED_LINE):
        _check(t, coords, vals, spec.dims, A, 64, variant, 8)
    _check(t, coords, vals, spec.dims, A, 64, TILED, 4, bf16=True)


def test_count_tensor_small_modes():
    """The 200- and 24-row modes: every row is hot, all updates staged."""
    spec = synth.scaled(synth.COUNT4D, 2_000_000)
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.rand_factors(spec.dims, 16, 6)
    _check(t, coords, vals, spec.dims, A, 16, TILED, 8)
    _check(t, coords, vals, spec.dims, A, 16, TILED_LINE, 4, modes=[2, 3])


def test_generic_kernel_six_and_two_modes():
    for dims in [(40, 30, 20, 10, 8, 6), (500, 300)]:
        coords, vals = gu.rand_tensor(dims, 30_000, len(dims))
        t = gu.encode(coords, vals, dims)
        A = gu.rand_factors(dims, 16, 7)
        _check(t, coords, vals, dims, A, 16, TILED, 8)
        _check(t, coords, vals, dims, A, 16, TILED_LINE, 4)


def test_mode_of_length_one_and_one_mode():
    import torch
    dims = (1, 300, 7)
    coords, vals = gu.rand_tensor(dims, 20_000, 9)
    t = gu.encode(coords, vals, dims)
    A = gu.rand_factors(dims, 8, 8)
    _check(t, coords, vals, dims, A, 8, TILED, 8)
    coords, vals = gu.rand_tensor((64,), 3000, 8)
    t = gu.encode(coords, vals, (64,))
    t.set_mode_plan(0, TILED, 4)
    got = t.mttkrp(0, [None], 4).cpu().numpy()
    want = np.bincount(coords[0], weights=vals.astype(np.float64), minlength=64)
    np.testing.assert_allclose(got[:, 0], want, rtol=1e-5)


def test_all_ones_factors_give_slice_sums():
    import torch
    dims = (50, 40, 30, 20)
    coords, vals = gu.rand_tensor(dims, 30_000, 7)
    t = gu.encode(coords, vals, dims)
    ones = [torch.ones((d, 8), device="cuda") for d in dims]
    for n in range(4):
        t.set_mode_plan(n, TILED, 8)
        got = t.mttkrp(n, ones, 8).cpu().numpy()
        want = np.bincount(coords[n], weights=vals.astype(np.float64), minlength=dims[n])
        for r in range(8):
            np.testing.assert_allclose(got[:, r], want, rtol=1e-5)


def test_empty_tensor_gives_zeros():
    import torch
    t = gu.encode(np.zeros((3, 0), np.uint32), np.zeros(0, np.float32), (10, 20, 30))
    t.set_mode_plan(1, TILED, 8)
    A = [torch.rand((d, 8), device="cuda") for d in (10, 20, 30)]
    out = torch.full((20, 8), 7.0, device="cuda")
    t.mttkrp(1, A, 8, out=out)
    assert float(out.abs().max()) == 0.0


def test_misaligned_factors_use_four_columns():
    """8 fp32 columns per lane need 32-byte aligned rows; a 16-byte aligned
    factor falls back to 4 columns per lane and stays correct."""
    import torch
    dims = (200, 150, 100)
    coords, vals = gu.rand_tensor(dims, 30_000, 4)
    t = gu.encode(coords, vals, dims)
    A = gu.rand_factors(dims, 16, 9)
    Ad = gu.gpu_factors(A)
    for m in range(3):   # views starting 16 bytes into a buffer
        buf = torch.empty(dims[m] * 16 + 4, device="cuda")
        v = buf[4:].view(dims[m], 16)
        v.copy_(Ad[m])
        Ad[m] = v
    for n in range(3):
        t.set_mode_plan(n, TILED, 8)
        got = t.mttkrp(n, Ad, 16).cpu().numpy()
        err, bad = ar.row_relative_error(got, cref.mttkrp(coords, vals, dims, A, n, nthreads=4))
        assert bad == 0 and err <= TOL_F32
