"""Plain numpy oracle for CP-APR with multiplicative updates (test
infrastructure only; only tests/, __graft_entry__.smoke() and bench.py's CPU
legs may use it). Everything is fp64.

It follows the CP-APR MU algorithm (Alg. 2) and the model-update kernel Phi of
Alg. 5 in the order the paper states them:

  for each outer iteration k, for each mode n:
    S(i,r) = kappa where k > 1, A^(n)(i,r) < kappa_tol and Phi^(n)(i,r) > 1
             (Phi^(n) from the previous outer iteration), else 0
    B = (A^(n) + S) diag(lambda)
    Pi = the Khatri-Rao product of the other factors (only the rows of
         nonzeros are ever used: krp(x) = *_{m != n} A^(m)(i_m(x), :))
    repeat at most l_max times:
      Phi^(n) = (X_(n) ./ max(B Pi, eps)) Pi^T, i.e. for every nonzero x
                Phi(i_n,:) += v_x / max(B(i_n,:) . krp(x), eps) * krp(x)
      stop when |min(B, E - Phi)| < tau
      B = B .* Phi
    lambda = e^T B (column sums), A^(n) = B diag(lambda)^-1
  stop when no mode took an update step in this outer iteration.

Readings (the paper gives no values and leaves one norm unnamed; each is also
restated in the design notes):

* |min(B, E - Phi)| is the largest absolute entry of the elementwise minimum
  (the KKT violation of the Poisson subproblem).
* kappa = 1e-2, kappa_tol = 1e-10, eps = 1e-10, tau = 1e-4 are the defaults;
  l_max = 10 is the value the paper uses (Section V-A).
* The initial guess is normalised first: each factor's columns are scaled to
  sum to 1 and lambda holds the products of the scales, so the model
  sum_r lambda_r a_r^(1) o ... o a_r^(N) is the one the caller passed.
* A column whose sum is 0 keeps lambda_r = 0 and is left as it is.
* Duplicate coordinates are separate entries of X_(n) that add into one cell;
  Phi sums their terms like any other nonzeros.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

DEFAULTS = dict(l_max=10, tau=1e-4, kappa=1e-2, kappa_tol=1e-10, eps=1e-10)


def krp_rows(coords: np.ndarray, A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """krp(x) = *_{m != n} A^(m)(i_m(x), :) for every nonzero x (rows of Pi^T)."""
    M = coords.shape[1]
    R = A[0].shape[1]
    K = np.ones((M, R))
    for m in range(len(A)):
        if m != n:
            K *= np.asarray(A[m], dtype=np.float64)[coords[m]]
    return K


def phi(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int], A: Sequence[np.ndarray],
        B: np.ndarray, n: int, eps: float = DEFAULTS["eps"]) -> np.ndarray:
    """Phi^(n) of Alg. 5: every nonzero adds v / max(B(i_n,:) . krp, eps) * krp
    to row i_n."""
    K = krp_rows(coords, A, n)
    rows = coords[n].astype(np.int64)
    denom = np.maximum(np.sum(np.asarray(B, dtype=np.float64)[rows] * K, axis=1), eps)
    contrib = (np.asarray(vals, dtype=np.float64) / denom)[:, None] * K
    out = np.zeros((dims[n], K.shape[1]))
    np.add.at(out, rows, contrib)
    return out


def poisson_objective(coords: np.ndarray, vals: np.ndarray, lam: np.ndarray,
                      A: Sequence[np.ndarray]) -> float:
    """f(M) = sum over all cells of M - sum over nonzeros of x log M(x), the
    negative Poisson log-likelihood up to a constant; sum over all cells of M
    is sum_r lambda_r prod_m sum_i A^(m)(i, r)."""
    lam = np.asarray(lam, dtype=np.float64)
    total = float(np.sum(lam * np.prod([np.asarray(a).sum(axis=0) for a in A], axis=0)))
    K = krp_rows(coords, A, -1)
    m = K @ lam
    with np.errstate(divide="ignore"):
        logm = np.log(np.maximum(m, 1e-300))
    return total - float(np.sum(np.asarray(vals, dtype=np.float64) * logm))


def normalize(init: Sequence[np.ndarray]):
    """Column-stochastic factors and the lambda that keeps the model."""
    A = [np.asarray(a, dtype=np.float64).copy() for a in init]
    R = A[0].shape[1]
    lam = np.ones(R)
    for a in A:
        s = a.sum(axis=0)
        nz = s > 0
        a[:, nz] /= s[nz]
        lam *= np.where(nz, s, 0.0)
    return lam, A


@dataclasses.dataclass
class APRResult:
    factors: List[np.ndarray]
    lam: np.ndarray
    objective: List[float]       # after every outer iteration
    inner: List[List[int]]       # update steps taken per mode, per outer iteration
    outer_done: int
    converged: bool


def cp_apr_mu(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int],
              init: Sequence[np.ndarray], k_max: int, l_max: int = DEFAULTS["l_max"],
              tau: float = DEFAULTS["tau"], kappa: float = DEFAULTS["kappa"],
              kappa_tol: float = DEFAULTS["kappa_tol"], eps: float = DEFAULTS["eps"],
              phi_fn=None) -> APRResult:
    """Alg. 2 (CP-APR, multiplicative updates) in fp64."""
    if phi_fn is None:
        phi_fn = phi
    N = len(dims)
    lam, A = normalize(init)
    R = lam.shape[0]
    phi_prev = [np.zeros((dims[n], R)) for n in range(N)]
    objective: List[float] = []
    inner: List[List[int]] = []
    converged = False
    k_done = 0
    for k in range(k_max):
        converged = True
        steps = []
        for n in range(N):
            S = np.where((k > 0) & (A[n] < kappa_tol) & (phi_prev[n] > 1.0), kappa, 0.0)
            B = (A[n] + S) * lam[None, :]
            taken = 0
            Phi = None
            for _ in range(l_max):
                Phi = phi_fn(coords, vals, dims, A, B, n, eps)
                if np.max(np.abs(np.minimum(B, 1.0 - Phi))) < tau:
                    break
                converged = False
                B = B * Phi
                taken += 1
            phi_prev[n] = Phi
            lam = B.sum(axis=0)
            nz = lam > 0
            A[n] = B.copy()
            A[n][:, nz] /= lam[nz]
            steps.append(taken)
        inner.append(steps)
        objective.append(poisson_objective(coords, vals, lam, A))
        k_done = k + 1
        if converged:
            break
    return APRResult(A, lam, objective, inner, k_done, converged)
