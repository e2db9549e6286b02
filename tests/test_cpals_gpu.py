"""GPU CP-ALS (Alg. 1) through the C ABI against the fp64 oracle.

MTTKRP parity is the hard gate; CP-ALS is a trajectory check: the fit after
every iteration within 1e-4 of the oracle's, columns normalised, exact low-rank
tensors recovered.
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _oracle_cpals(coords, vals, dims, init, iters, tol=0.0):
    return ar.cp_als(coords, vals, dims, init, iters, tol=tol)


@pytest.mark.parametrize("R", [4, 8, 16, 32, 64])
def test_fit_trajectory_matches_oracle(R):
    spec = synth.scaled(synth.UNIFORM3D, 20_000, dims=(200, 160, 120))
    coords, vals = synth.generate(spec)
    init = gu.rand_factors(spec.dims, R, 3)
    ref = _oracle_cpals(coords, vals, spec.dims, init, iters=6)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.gpu_factors(init)
    lam, fits = t.cpals(R, 6, A)
    assert len(fits) == 6
    np.testing.assert_allclose(fits, ref.fits, atol=1e-4)
    for a in A:
        np.testing.assert_allclose(a.norm(dim=0).cpu().numpy(), 1.0, rtol=1e-4)
    np.testing.assert_allclose(lam, ref.lam, rtol=1e-2)


def test_fit_trajectory_zipf_skewed():
    """Zipf heads make the columns of M nearly collinear in early iterations;
    the fit and lambda must still follow the fp64 oracle."""
    spec = synth.scaled(synth.ZIPF3D, 300_000, dims=(200_000, 40_000, 5_000))
    coords, vals = synth.generate(spec)
    R = 16
    init = gu.rand_factors(spec.dims, R, 11)
    ref = _oracle_cpals(coords, vals, spec.dims, init, iters=4)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.gpu_factors(init)
    lam, fits = t.cpals(R, 4, A)
    np.testing.assert_allclose(fits, ref.fits, atol=1e-4)
    np.testing.assert_allclose(np.sort(lam), np.sort(ref.lam), rtol=1e-2)


def test_exact_low_rank_recovered():
    """An exact rank-4 tensor decomposed at R = 4 reaches fit 1 (up to fp32)."""
    rng = np.random.default_rng(1)
    dims, R = (60, 50, 40), 4
    F = [np.abs(rng.standard_normal((d, R))) * (rng.random((d, 1)) < 0.6) for d in dims]
    X = ar.reconstruct_dense(np.ones(R), F)
    nz = np.nonzero(X)
    coords = np.stack(nz).astype(np.uint32)
    vals = X[nz].astype(np.float32)
    t = gu.encode(coords, vals, dims)
    A = gu.gpu_factors([np.random.default_rng(2).random((d, R)).astype(np.float32) for d in dims])
    lam, fits = t.cpals(R, 150, A)
    # The fit is evaluated from fp32 MTTKRP output through the expansion
    # ||X||^2 + ||X_hat||^2 - 2<X, X_hat>, whose cancellation limits it to about
    # sqrt(fp32 epsilon) near 1; the model itself is checked directly in fp64.
    assert fits[-1] > 1 - 1e-3
    Xh = ar.reconstruct_dense(lam, [a.double().cpu().numpy() for a in A])
    assert np.linalg.norm(X - Xh) / np.linalg.norm(X) < 1e-4


def test_tol_stops_early_and_host_factors_match_device():
    spec = synth.scaled(synth.UNIFORM3D, 10_000, dims=(100, 90, 80))
    coords, vals = synth.generate(spec)
    init = gu.rand_factors(spec.dims, 8, 5)
    t = gu.encode(coords, vals, spec.dims)
    Ad = gu.gpu_factors(init)
    lam_d, fits_d = t.cpals(8, 50, Ad, tol=1e-3)
    assert 1 < len(fits_d) < 50
    assert abs(fits_d[-1] - fits_d[-2]) < 1e-3
    Ah = [a.copy() for a in init]
    lam_h, fits_h = t.cpals(8, 50, Ah, tol=1e-3)
    assert len(fits_h) == len(fits_d)
    np.testing.assert_allclose(fits_h, fits_d, atol=1e-5)
    for a, b in zip(Ah, Ad):
        np.testing.assert_allclose(a, b.cpu().numpy(), atol=1e-4)


def test_singular_gram_falls_back_to_pinv():
    """A zero column in every factor makes V singular: the solve uses the
    pseudo-inverse (fp64 Jacobi on the GPU, numpy's pinv in the oracle) and the
    trajectory still follows the oracle; the zero column stays zero."""
    dims = (30, 20, 10)
    coords, vals = gu.rand_tensor(dims, 2000, 4)
    t = gu.encode(coords, vals, dims)
    init = gu.rand_factors(dims, 4, 6)
    for a in init:
        a[:, 1] = 0.0          # a zero column in every factor: V has a zero pivot
    ref = _oracle_cpals(coords, vals, dims, init, iters=3)
    A = gu.gpu_factors(init)
    lam, fits = t.cpals(4, 3, A)
    np.testing.assert_allclose(fits, ref.fits, atol=1e-4)
    for a in A:
        assert float(a[:, 1].abs().max()) == 0.0


def test_non_finite_factors_report_not_spd():
    import paper_2403_06348_gb300 as alto
    dims = (30, 20, 10)
    coords, vals = gu.rand_tensor(dims, 2000, 4)
    t = gu.encode(coords, vals, dims)
    init = gu.rand_factors(dims, 4, 6)
    init[2][3, 1] = np.nan
    A = gu.gpu_factors(init)
    with pytest.raises(alto.AltoError) as e:
        t.cpals(4, 3, A)
    assert e.value.status == -6
    # the handle stays usable
    A2 = gu.gpu_factors(gu.rand_factors(dims, 4, 7))
    t.cpals(4, 2, A2)


@pytest.mark.slow
def test_full_size_first_iteration_fit():
    """Iteration 1 of Alg. 1 (every mode update, then the fit) on the
    1e8-nonzero Zipf tensor 10M x 2M x 50k at R = 32, the bench's workload:
    the GPU's fit equals the oracle's (fp64 solve, C fp64 MTTKRP) within 1e-4."""
    import os
    from oracle import cref
    spec = synth.ZIPF3D
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    init = synth.factors(spec.dims, spec.rank, seed=1)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.gpu_factors(init)
    _, fits = t.cpals(spec.rank, 1, A)
    t.free()
    del A
    nt = os.cpu_count() or 1
    ref = ar.cp_als(coords, vals, spec.dims, init, 1,
                    mttkrp_fn=lambda c, v, F, n: cref.mttkrp(c, v, spec.dims, F, n, nthreads=nt))
    assert abs(fits[0] - ref.fits[0]) <= 1e-4, (fits[0], ref.fits[0])
