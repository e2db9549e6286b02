"""GPU MTTKRP parity through the C ABI against the fp64 oracle.

Bar (row-relative error, max over rows of ||got_i - ref_i||_inf / ||ref_i||_inf):
fp32 factors <= 1e-5; bf16 factors <= 1e-2 against the oracle run on the
original fp32 factors (so the bf16 rounding is counted). Rows the oracle
leaves empty must be exactly 0.
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


def _run_modes(coords, vals, dims, R, variant=0, cpl=0, bf16=False, seed=0, modes=None,
               factors=None, tol=None):
    import torch
    import paper_2403_06348_gb300 as alto
    t = gu.encode(coords, vals, dims)
    A = factors if factors is not None else gu.rand_factors(dims, R, seed)
    Ad = gu.gpu_factors(A, torch.bfloat16 if bf16 else torch.float32)
    worst = 0.0
    for n in (modes if modes is not None else range(len(dims))):
        t.set_mode_plan(n, variant, cpl)
        got = t.mttkrp(n, Ad, R).cpu().numpy()
        ref = cref.mttkrp(coords, vals, dims, A, n, nthreads=4)
        err, bad_zero = ar.row_relative_error(got, ref)
        assert bad_zero == 0, f"mode {n}: rows without nonzeros are not exactly 0"
        limit = tol if tol is not None else (TOL_BF16 if bf16 else TOL_F32)
        assert err <= limit, f"mode {n}: row-relative error {err:.3g} > {limit}"
        worst = max(worst, err)
    return t, worst


# cols_per_lane: 4 and 8 split a nonzero over R/4 or R/8 lanes; 16 (= R here)
# is the one-thread-per-nonzero kernel
@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("cpl", [4, 8, 16])
def test_uniform_3d_all_modes(variant, cpl):
    spec = synth.UNIFORM3D
    coords, vals = synth.generate(spec)
    _run_modes(coords, vals, spec.dims, spec.rank, variant=variant, cpl=cpl, seed=1)


@pytest.mark.parametrize("R", [4, 8, 16, 32, 64])
@pytest.mark.parametrize("one_thread", [False, True])
def test_ranks(R, one_thread):
    coords, vals = gu.rand_tensor((300, 200, 150), 40_000, 3)
    _run_modes(coords, vals, (300, 200, 150), R, seed=R, cpl=R if one_thread else 0)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("cpl", [4, 16])
def test_bf16_factors(variant, cpl):
    spec = synth.UNIFORM3D
    coords, vals = synth.generate(spec)
    _run_modes(coords, vals, spec.dims, 16, variant=variant, cpl=cpl, bf16=True, seed=2)


@pytest.mark.parametrize("cpl", [4, 64])
def test_five_modes_two_word_positions(cpl):
    spec = synth.scaled(synth.ZIPF5D, 300_000)
    coords, vals = synth.generate(spec)
    _run_modes(coords, vals, spec.dims, 64, cpl=cpl, seed=4)
    _run_modes(coords, vals, spec.dims, 64, cpl=cpl, bf16=True, seed=4)


@pytest.mark.parametrize("cpl", [4, 8, 32])
def test_zipf_hot_rows(cpl):
    spec = synth.scaled(synth.ZIPF3D, 2_000_000)
    coords, vals = synth.generate(spec)
    _run_modes(coords, vals, spec.dims, 32, variant=1, seed=5, cpl=cpl)


def test_six_and_two_modes_generic_kernel():
    """N outside {3, 4, 5} runs the kernel with a run-time number of modes."""
    for dims in [(40, 30, 20, 10, 8, 6), (500, 300)]:
        coords, vals = gu.rand_tensor(dims, 30_000, len(dims))
        _run_modes(coords, vals, dims, 16, seed=7)
        _run_modes(coords, vals, dims, 16, seed=7, cpl=16)


def test_count_tensor_small_modes_pull():
    spec = synth.scaled(synth.COUNT4D, 2_000_000)
    coords, vals = synth.generate(spec)
    t, _ = _run_modes(coords, vals, spec.dims, 16, seed=6)
    assert t.get_mode_plan(3, 16)[0] == 3   # AUTO: the stored output-oriented order
    # the recursive traversal on the 200- and 24-row modes (reuse 10k, 83k)
    _run_modes(coords, vals, spec.dims, 16, variant=2, seed=6, modes=[2, 3])
    _run_modes(coords, vals, spec.dims, 16, variant=2, seed=6, modes=[2, 3])
    _run_modes(coords, vals, spec.dims, 16, variant=2, seed=6, modes=[2, 3], cpl=16)
    _run_modes(coords, vals, spec.dims, 16, variant=1, seed=6, modes=[2, 3])


def test_all_ones_factors_give_slice_sums():
    import torch
    dims = (50, 40, 30, 20)
    coords, vals = gu.rand_tensor(dims, 30_000, 7)
    t = gu.encode(coords, vals, dims)
    ones = [torch.ones((d, 8), device="cuda") for d in dims]
    for n in range(4):
        got = t.mttkrp(n, ones, 8).cpu().numpy()
        want = np.bincount(coords[n], weights=vals.astype(np.float64), minlength=dims[n])
        for r in range(8):
            np.testing.assert_allclose(got[:, r], want, rtol=1e-5)


def test_empty_tensor_gives_zeros():
    import torch
    t = gu.encode(np.zeros((3, 0), np.uint32), np.zeros(0, np.float32), (10, 20, 30))
    A = [torch.rand((d, 8), device="cuda") for d in (10, 20, 30)]
    out = torch.full((20, 8), 7.0, device="cuda")
    t.mttkrp(1, A, 8, out=out)
    assert float(out.abs().max()) == 0.0


def test_one_mode_tensor():
    import torch
    coords, vals = gu.rand_tensor((64,), 500, 8)
    t = gu.encode(coords, vals, (64,))
    got = t.mttkrp(0, [None], 4).cpu().numpy()
    want = np.bincount(coords[0], weights=vals.astype(np.float64), minlength=64)
    np.testing.assert_allclose(got[:, 0], want, rtol=1e-5)


def test_bad_arguments_rejected():
    import torch
    import paper_2403_06348_gb300 as alto
    coords, vals = gu.rand_tensor((10, 10, 10), 100, 1)
    t = gu.encode(coords, vals, (10, 10, 10))
    A = [torch.rand((10, 16), device="cuda") for _ in range(3)]
    with pytest.raises(alto.AltoError) as e:
        t.mttkrp(3, A, 16)
    assert e.value.status == -1
    with pytest.raises(alto.AltoError) as e:
        t.mttkrp(0, [torch.rand((10, 12), device="cuda")] * 3, 12)
    assert e.value.status == -4
    with pytest.raises(alto.AltoError):
        t.mttkrp(0, [A[0], None, A[2]], 16)


# ---------------------------------------------------------------------------
# full-size workloads: sampled rows (the hottest rows, random rows) against
# the fp64 oracle computed row by row
# ---------------------------------------------------------------------------

def _full_size_rows(spec, R, bf16=False, nrand=192, nhot=64, seed=10, variant=0):
    import torch
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.rand_factors(spec.dims, R, seed)
    Ad = gu.gpu_factors(A, torch.bfloat16 if bf16 else torch.float32)
    rng = np.random.default_rng(seed)
    for n in range(len(spec.dims)):
        t.set_mode_plan(n, variant)
        got = t.mttkrp(n, Ad, R)
        counts = np.bincount(coords[n], minlength=spec.dims[n])
        hot = np.argsort(-counts, kind="stable")[:nhot]
        rnd = rng.choice(spec.dims[n], size=min(nrand, spec.dims[n]), replace=False)
        empty = np.nonzero(counts == 0)[0][:64]
        rows = np.unique(np.concatenate([hot, rnd, empty])).astype(np.uint32)
        ref = cref.mttkrp_rows(coords, vals, spec.dims, A, n, rows)
        g = got[torch.from_numpy(rows.astype(np.int64)).cuda()].cpu().numpy()
        err, bad_zero = ar.row_relative_error(g, ref)
        assert bad_zero == 0
        assert err <= (TOL_BF16 if bf16 else TOL_F32), f"mode {n}: {err:.3g}"
        del got
    t.free()


@pytest.mark.slow
@pytest.mark.parametrize("variant", [0, 4])
def test_full_size_zipf3d(variant):
    _full_size_rows(synth.ZIPF3D, 32, variant=variant)


@pytest.mark.slow
@pytest.mark.parametrize("variant", [0, 4])
def test_full_size_count4d(variant):
    _full_size_rows(synth.COUNT4D, 16, variant=variant)


@pytest.mark.slow
@pytest.mark.parametrize("variant", [0, 4])
def test_full_size_zipf5d_fp32_and_bf16(variant):
    _full_size_rows(synth.ZIPF5D, 64, variant=variant)
    _full_size_rows(synth.ZIPF5D, 64, bf16=True, variant=variant)
