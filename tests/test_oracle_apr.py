"""Pins of the CP-APR oracle (oracle/apr_ref.py) against what the mathematics
fixes: the dense unfolded form of Phi, the fixed point of an exact model, the
closed-form rank-1 solution, the Poisson objective by brute force, monotone
descent, and the inadmissible-zero shift."""
import numpy as np
import pytest

from oracle import alto_ref as ar
from oracle import apr_ref as apr


def _counts(dims, M, seed):
    rng = np.random.default_rng(seed)
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    vals = (rng.poisson(3.0, M) + 1).astype(np.float64)
    return coords, vals


def _rand(dims, R, seed, lo=0.1):
    rng = np.random.default_rng(seed)
    return [lo + rng.random((d, R)) for d in dims]


@pytest.mark.parametrize("dims,R", [((5, 4, 3), 3), ((4, 3, 5, 2), 2), ((6, 7), 4)])
def test_phi_equals_dense_unfolded_form(dims, R):
    """Phi = (X_(n) ./ max(B Pi, eps)) Pi^T with the explicit unfolding and an
    explicit Khatri-Rao product; duplicates included."""
    coords, vals = _counts(dims, 40, 1)
    coords[:, 5] = coords[:, 3]  # a duplicate coordinate
    A = _rand(dims, R, 2)
    X = ar.to_dense(coords, vals, dims)
    for n in range(len(dims)):
        B = _rand([dims[n]], R, 3 + n)[0]
        others = [A[m] for m in range(len(dims)) if m != n]
        Pi = ar.khatri_rao(others, R)                   # J x R
        dense = (ar.unfold(X, n) / np.maximum(B @ Pi.T, 1e-10)) @ Pi
        np.testing.assert_allclose(apr.phi(coords, vals, dims, A, B, n), dense, rtol=1e-12)


def test_objective_equals_brute_force():
    dims, R = (4, 5, 3), 3
    coords, vals = _counts(dims, 30, 4)
    lam, A = apr.normalize(_rand(dims, R, 5))
    X = ar.to_dense(coords, vals, dims)
    Mdl = ar.reconstruct_dense(lam, A)
    brute = float(Mdl.sum() - np.sum(X[X > 0] * np.log(Mdl[X > 0])))
    assert apr.poisson_objective(coords, vals, lam, A) == pytest.approx(brute, rel=1e-12)


def test_exact_model_is_a_fixed_point():
    """X equal to a positive model with column-stochastic factors: every Phi is
    all ones (the KKT conditions hold), so CP-APR stops at once and returns
    the model."""
    dims, R = (4, 3, 5), 2
    lam, A = apr.normalize(_rand(dims, R, 6, lo=0.5))
    X = ar.reconstruct_dense(lam, A)
    coords = np.stack(np.nonzero(X > -1)).astype(np.uint32)   # every cell
    vals = X[tuple(coords)]
    for n in range(3):
        Phi = apr.phi(coords, vals, dims, A, A[n] * lam[None, :], n)
        np.testing.assert_allclose(Phi, 1.0, rtol=1e-12)
    init = [A[0] * lam[None, :]] + [a.copy() for a in A[1:]]   # the model itself
    res = apr.cp_apr_mu(coords, vals, dims, init, k_max=5)
    assert res.converged and res.outer_done == 1 and res.inner == [[0, 0, 0]]


def test_rank_one_gives_the_marginals():
    """At R = 1 the Poisson MLE given the other factors is the mode-n marginal
    of X: after one outer iteration every factor is its normalised marginal,
    lambda is the total count, and the second iteration takes no step."""
    dims = (6, 5, 4)
    coords, vals = _counts(dims, 50, 7)
    res = apr.cp_apr_mu(coords, vals, dims, _rand(dims, 1, 8), k_max=10)
    total = vals.sum()
    assert res.lam[0] == pytest.approx(total, rel=1e-10)
    for n in range(3):
        marg = np.bincount(coords[n], weights=vals, minlength=dims[n]) / total
        np.testing.assert_allclose(res.factors[n][:, 0], marg, rtol=1e-9, atol=1e-14)
    assert res.converged and res.outer_done == 2 and res.inner[1] == [0, 0, 0]


def test_objective_never_increases():
    dims, R = (20, 15, 10), 4
    coords, vals = _counts(dims, 400, 9)
    res = apr.cp_apr_mu(coords, vals, dims, _rand(dims, R, 10), k_max=15)
    f = np.array(res.objective)
    assert np.all(np.diff(f) <= 1e-9 * np.abs(f[:-1]))
    assert f[-1] < f[0]


def test_inadmissible_zero_shift_lets_a_zero_entry_grow():
    """Multiplicative updates keep an exact zero at zero; the kappa shift moves
    entries below kappa_tol whose Phi exceeds 1 off zero, and the fit gets
    better than with the shift turned off."""
    dims, R = (6, 5, 4), 2
    lam0, A0 = apr.normalize(_rand(dims, R, 11, lo=0.3))
    X = ar.reconstruct_dense(lam0, A0)
    coords = np.stack(np.nonzero(X > -1)).astype(np.uint32)
    vals = X[tuple(coords)]
    init = [a.copy() for a in _rand(dims, R, 12, lo=0.3)]
    init[0][2, 1] = 0.0          # the model needs this entry positive
    off = apr.cp_apr_mu(coords, vals, dims, init, k_max=60, kappa=0.0)
    on = apr.cp_apr_mu(coords, vals, dims, init, k_max=60)
    assert off.factors[0][2, 1] == 0.0
    assert on.factors[0][2, 1] > 1e-3
    assert on.objective[-1] < off.objective[-1]
