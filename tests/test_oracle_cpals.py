"""Pins for the oracle's CP-ALS (Alg. 1).

Checked against least squares solved by numpy.linalg.lstsq on the dense
unfolding, a direct dense evaluation of ||X - X_hat||, exact low-rank
recovery, and the monotone fit of alternating least squares.
"""
import numpy as np
import pytest

from oracle import alto_ref as ar


def _sparse_low_rank(dims, R, density, seed):
    rng = np.random.default_rng(seed)
    F = [np.abs(rng.standard_normal((d, R))) * (rng.random((d, 1)) < density) for d in dims]
    X = ar.reconstruct_dense(np.ones(R), F)
    nz = np.nonzero(X)
    coords = np.stack(nz).astype(np.uint32)
    vals = X[nz].astype(np.float32)
    return coords, vals, X


def test_single_update_is_least_squares():
    """One mode update of Alg. 1 (before normalisation) minimises
    ||X_(n) - A K^T|| over A: compare with lstsq on the dense unfolding."""
    rng = np.random.default_rng(0)
    dims, R = (6, 5, 4), 3
    M = 60
    flat = rng.choice(np.prod(dims), M, replace=False)
    coords = np.stack(np.unravel_index(flat, dims)).astype(np.uint32)
    vals = rng.standard_normal(M).astype(np.float32)
    A = [rng.standard_normal((d, R)) for d in dims]
    X = ar.to_dense(coords, vals, dims)
    n = 1
    V = np.ones((R, R))
    for m in range(3):
        if m != n:
            V *= A[m].T @ A[m]
    An = ar._solve_spd_or_pinv(V, ar.mttkrp(coords, vals, A, n))
    K = ar.khatri_rao([A[m] for m in range(3) if m != n])
    ls = np.linalg.lstsq(K, ar.unfold(X, n).T, rcond=None)[0].T
    np.testing.assert_allclose(An, ls, rtol=1e-9, atol=1e-10)


def test_fit_matches_dense_residual():
    rng = np.random.default_rng(1)
    dims, R = (5, 4, 6), 2
    coords, vals, _ = _sparse_low_rank(dims, 3, 0.8, seed=2)
    init = [rng.random((d, R)) for d in dims]
    res = ar.cp_als(coords, vals, dims, init, iters=3)
    X = ar.to_dense(coords, vals, dims)
    Xh = ar.reconstruct_dense(res.lam, res.factors)
    direct = 1 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
    assert abs(direct - res.fits[-1]) < 1e-10


def test_norm_and_fit_with_duplicate_coordinates():
    """Duplicates add up into one cell: ||X||^2 and the fit follow the dense
    tensor built with np.add.at."""
    rng = np.random.default_rng(3)
    dims, R = (5, 4, 3), 2
    M = 200
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    vals = rng.random(M).astype(np.float32)
    X = ar.to_dense(coords, vals, dims)
    assert abs(ar.tensor_norm_sq(coords, vals) - np.sum(X * X)) < 1e-9 * np.sum(X * X)
    assert ar.tensor_norm_sq(coords, vals) > 1.5 * np.sum(vals.astype(np.float64) ** 2)
    init = [rng.random((d, R)) for d in dims]
    res = ar.cp_als(coords, vals, dims, init, iters=4)
    Xh = ar.reconstruct_dense(res.lam, res.factors)
    direct = 1 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
    assert abs(direct - res.fits[-1]) < 1e-10


@pytest.mark.parametrize("R", [1, 2])
def test_exact_low_rank_recovered(R):
    dims = (8, 7, 6)
    coords, vals, _ = _sparse_low_rank(dims, R, 0.6, seed=10 + R)
    rng = np.random.default_rng(4)
    init = [rng.random((d, R)) for d in dims]
    res = ar.cp_als(coords, vals, dims, init, iters=500)
    assert res.fits[-1] > 1 - 1e-6


def test_fit_monotone_non_decreasing():
    rng = np.random.default_rng(6)
    dims = (30, 25, 20)
    M = 800
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    vals = rng.random(M).astype(np.float32) + 0.1
    init = [rng.random((d, 4)) for d in dims]
    res = ar.cp_als(coords, vals, dims, init, iters=15)
    f = np.array(res.fits)
    assert np.all(np.diff(f) >= -1e-10)


def test_columns_normalised_and_tol_stops_early():
    rng = np.random.default_rng(8)
    dims = (12, 10, 9)
    coords, vals, _ = _sparse_low_rank(dims, 2, 0.7, seed=3)
    init = [rng.random((d, 3)) for d in dims]
    res = ar.cp_als(coords, vals, dims, init, iters=100, tol=1e-3)
    for A in res.factors:
        np.testing.assert_allclose(np.linalg.norm(A, axis=0), 1.0, rtol=1e-12)
    assert len(res.fits) < 100


def test_singular_gram_uses_pinv():
    """Identical columns make V singular; Alg. 1's pseudo-inverse still gives
    the minimum-norm least-squares update."""
    rng = np.random.default_rng(2)
    dims = (6, 5, 4)
    M = 40
    flat = rng.choice(np.prod(dims), M, replace=False)
    coords = np.stack(np.unravel_index(flat, dims)).astype(np.uint32)
    vals = rng.random(M).astype(np.float32)
    col = [rng.random((d, 1)) for d in dims]
    A = [np.hstack([c, c]) for c in col]
    V = (A[1].T @ A[1]) * (A[2].T @ A[2])
    M0 = ar.mttkrp(coords, vals, A, 0)
    An = ar._solve_spd_or_pinv(V, M0)
    assert np.all(np.isfinite(An))
    np.testing.assert_allclose(An[:, 0], An[:, 1], rtol=1e-9)


def test_zero_column_stays_exactly_zero_through_pinv():
    """A zero column in every initial factor makes every V singular; the pinv
    solution leaves that column at rounding level, which the normalisation
    reads as zero: the column stays exactly 0 with lambda 0, and the other
    columns match a rank-(R-1) run without it."""
    rng = np.random.default_rng(21)
    dims = (12, 9, 7)
    coords = np.stack([rng.integers(0, d, 300) for d in dims]).astype(np.uint32)
    vals = rng.random(300)
    init = [rng.random((d, 3)) for d in dims]
    padded = [np.insert(a, 1, 0.0, axis=1) for a in init]
    full = ar.cp_als(coords, vals, dims, padded, 4)
    small = ar.cp_als(coords, vals, dims, init, 4)
    np.testing.assert_allclose(full.fits, small.fits, rtol=1e-9)
    assert full.lam[1] == 0.0
    for a, b in zip(full.factors, small.factors):
        assert np.all(a[:, 1] == 0.0)
        np.testing.assert_allclose(np.delete(a, 1, axis=1), b, rtol=1e-7, atol=1e-10)
