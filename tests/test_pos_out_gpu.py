"""The stored output-oriented order pos_out (Alg. 4) and the OUTPUT MTTKRP
through the C ABI.

pos_out must equal the oracle's bit for bit (a permutation of positions, so
integer work), for several segment counts, key widths and ragged sizes. The
OUTPUT MTTKRP meets the MTTKRP bar: row-relative error <= 1e-5 with fp32
factors and <= 1e-2 with bf16 factors against the fp64 oracle on the fp32
factors; rows without nonzeros exactly 0.
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from oracle import cref
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

OUTPUT = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _zipf(dims, nnz, seed):
    spec = synth.TensorSpec(f"po{seed}", tuple(dims), nnz, ("zipf:1.1",) * len(dims), "uniform01", 8,
                            seed=seed)
    return synth.generate(spec)


@pytest.mark.parametrize("dims,nnz,L", [((300, 200, 24), 40_000, 0), ((300, 200, 24), 40_000, 1),
                                         ((300, 200, 24), 40_001, 7), ((500, 400, 30, 12), 30_011, 0),
                                         ((2_000_000, 100_000, 10_000, 1000, 50), 30_000, 0),
                                         ((2_000_000, 100_000, 10_000, 1000, 50), 30_000, 30_000),
                                         ((50, 1, 40), 3_333, 5), ((7, 9, 5), 1, 0),
                                         # segments of 8192 (one CTA each) and 8193 (one sort)
                                         ((300, 200, 24), 16_384, 2), ((300, 200, 24), 16_385, 2),
                                         ((1_000_000, 3, 1000), 250_000, 0)])
def test_pos_out_equals_oracle(dims, nnz, L):
    coords, vals = _zipf(dims, nnz, 1 + nnz % 97)
    t = gu.encode(coords, vals, dims)
    ref_t = ar.encode(coords, vals, dims)
    Lused = L if L else max(int(t.query().nparts), -(-nnz // 8192))
    t.build_pos_out(-1, L)
    for n in range(len(dims)):
        got, Lgot = t.pos_out(n)
        assert Lgot == min(max(Lused, 1), nnz)
        want = ar.pos_out(ref_t, Lgot, n)
        np.testing.assert_array_equal(got.astype(np.int64), want)


def _check(t, coords, vals, dims, A, Ad, R, modes, tol):
    for n in modes:
        got = t.mttkrp(n, Ad, R).cpu().numpy()
        ref = cref.mttkrp(coords, vals, dims, A, n, nthreads=4)
        err, bad_zero = ar.row_relative_error(got, ref)
        assert bad_zero == 0, f"mode {n}: rows without nonzeros are not exactly 0"
        assert err <= tol, f"mode {n} R {R}: row-relative error {err:.3g} > {tol}"


@pytest.mark.parametrize("R", [4, 8, 16, 32, 64])
@pytest.mark.parametrize("cpl", [4, 8])
def test_output_mttkrp_ranks(R, cpl):
    dims = (300, 200, 150)
    coords, vals = _zipf(dims, 40_000 + R, 3)
    t = gu.encode(coords, vals, dims)
    A = gu.rand_factors(dims, R, R)
    Ad = gu.gpu_factors(A)
    for n in range(3):
        t.set_mode_plan(n, OUTPUT, cpl)
        assert t.get_mode_plan(n, R)[:2] == (OUTPUT, 8 if (cpl == 8 and R >= 8) else 4)
    _check(t, coords, vals, dims, A, Ad, R, range(3), 1e-5)


@pytest.mark.parametrize("L", [1, 13, 0])
def test_output_mttkrp_segment_counts_and_modes(L):
    import paper_2403_06348_gb300 as alto
    for dims, nnz in [((500, 400, 30, 12), 30_011), ((400, 300, 50, 20, 8), 25_000),
                      ((2_000_000, 100_000, 10_000, 1000, 50), 30_000),
                      ((40, 30, 20, 10, 8, 6), 9_000)]:
        coords, vals = _zipf(dims, nnz, 5)
        t = gu.encode(coords, vals, dims)
        t.build_pos_out(-1, L)
        A = gu.rand_factors(dims, 16, 6)
        Ad = gu.gpu_factors(A)
        for n in range(len(dims)):
            t.set_mode_plan(n, alto.VARIANT_OUTPUT, 4)
        _check(t, coords, vals, dims, A, Ad, 16, range(len(dims)), 1e-5)


@pytest.mark.parametrize("cpl", [4, 8])
def test_output_mttkrp_bf16(cpl):
    import torch
    spec = synth.UNIFORM3D
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.rand_factors(spec.dims, 16, 2)
    Ad = gu.gpu_factors(A, torch.bfloat16)
    for n in range(len(spec.dims)):
        t.set_mode_plan(n, OUTPUT, cpl)
    _check(t, coords, vals, spec.dims, A, Ad, 16, range(len(spec.dims)), 1e-2)


def test_output_built_on_first_use_and_freed():
    dims = (120, 90, 70)
    coords, vals = _zipf(dims, 5_000, 8)
    t = gu.encode(coords, vals, dims)
    import paper_2403_06348_gb300 as alto
    with pytest.raises(alto.AltoError):
        t.pos_out(0)                       # nothing stored yet
    A = gu.rand_factors(dims, 8, 9)
    Ad = gu.gpu_factors(A)
    before = t.query().device_bytes
    t.build_pos_out(1)
    # mode 1's order: positions (4 B), line positions (8 B) and values (4 B) per nonzero
    assert t.query().device_bytes == before + 16 * 5_000
    t.free_pos_out(1)
    assert t.query().device_bytes == before
    t.set_mode_plan(1, OUTPUT, 4)
    _check(t, coords, vals, dims, A, Ad, 8, [1], 1e-5)   # built on first use
    got, L = t.pos_out(1)
    np.testing.assert_array_equal(got.astype(np.int64), ar.pos_out(ar.encode(coords, vals, dims), L, 1))
    # the stored order does not follow later re-partitioning
    t.set_partitions(3)
    got2, L2 = t.pos_out(1)
    assert L2 == L
    np.testing.assert_array_equal(got2, got)
    _check(t, coords, vals, dims, A, Ad, 8, [1], 1e-5)
    held = t.query().device_bytes      # the re-partition changed the interval table's size
    t.free_pos_out(-1)
    assert t.query().device_bytes == held - 16 * 5_000
    _check(t, coords, vals, dims, A, Ad, 8, [1], 1e-5)   # rebuilt on use


def test_output_empty_and_single_nonzero():
    import paper_2403_06348_gb300 as alto
    dims = (30, 20, 10)
    coords = np.zeros((3, 0), dtype=np.uint32)
    vals = np.zeros(0, dtype=np.float32)
    t = gu.encode(coords, vals, dims)
    t.build_pos_out(-1)
    A = gu.rand_factors(dims, 8, 1)
    t.set_mode_plan(0, alto.VARIANT_OUTPUT, 4)
    out = t.mttkrp(0, gu.gpu_factors(A), 8).cpu().numpy()
    assert out.shape == (30, 8) and not out.any()
    coords1 = np.array([[29], [0], [9]], dtype=np.uint32)
    vals1 = np.array([2.5], dtype=np.float32)
    t1 = gu.encode(coords1, vals1, dims)
    for n in range(3):
        t1.set_mode_plan(n, OUTPUT, 4)
    _check(t1, coords1, vals1, dims, A, gu.gpu_factors(A), 8, range(3), 1e-6)


def test_autotune_with_output_candidates():
    dims = (5_000, 3_000, 200)
    coords, vals = _zipf(dims, 200_000, 11)
    t = gu.encode(coords, vals, dims)
    A = gu.rand_factors(dims, 32, 12)
    Ad = gu.gpu_factors(A)
    rep = t.autotune(Ad, 32, output=True)
    assert rep["candidates"] >= 3 * 4
    for n, (variant, _, _) in enumerate(rep["plans"]):
        if variant != OUTPUT:
            import paper_2403_06348_gb300 as alto
            with pytest.raises(alto.AltoError):
                t.pos_out(n)                 # the tuner's order is not kept
    _check(t, coords, vals, dims, A, Ad, 32, range(3), 1e-5)


def test_pos_out_bad_arguments():
    import paper_2403_06348_gb300 as alto
    dims = (30, 20, 10)
    coords, vals = _zipf(dims, 500, 13)
    t = gu.encode(coords, vals, dims)
    with pytest.raises(alto.AltoError):
        t.build_pos_out(3)
    with pytest.raises(alto.AltoError):
        t.build_pos_out(-2)
    with pytest.raises(alto.AltoError):
        t.free_pos_out(5)
