"""Pins for the oracle's MTTKRP (Alg. 1 MTTKRP line, Alg. 3).

The sparse definition is checked against the dense unfolding times an
explicit Khatri-Rao product (Section II-A notation), a closed form for rank-one
tensors, the all-ones slice-sum invariant, permutation invariance and exact
zeros for empty rows. The C oracle is checked against the same pins.
"""
import numpy as np
import pytest

from oracle import alto_ref as ar
from oracle import cref


def _random_tensor(dims, M, seed, dup=True):
    rng = np.random.default_rng(seed)
    if dup:
        coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    else:
        flat = rng.choice(int(np.prod(dims)), M, replace=False)
        coords = np.stack(np.unravel_index(flat, dims)).astype(np.uint32)
    vals = rng.standard_normal(M).astype(np.float32)
    return coords, vals


def _factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((d, R)).astype(np.float32) for d in dims]


@pytest.mark.parametrize("dims,M,R", [((4, 8, 2), 6, 3), ((5, 3, 4), 40, 2), ((3, 4, 2, 5), 60, 4),
                                       ((2, 3, 2, 3, 2), 50, 3), ((7, 6), 20, 5), ((9,), 12, 2),
                                       ((4, 1, 3), 10, 2)])
def test_sparse_equals_dense_unfolding(dims, M, R):
    coords, vals = _random_tensor(dims, M, seed=M + R)
    A = _factors(dims, R, seed=R)
    X = ar.to_dense(coords, vals, dims)
    for n in range(len(dims)):
        want = ar.mttkrp_dense(X, A, n)
        got = ar.mttkrp(coords, vals, A, n)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(cref.mttkrp(coords, vals, dims, A, n, nthreads=1), want,
                                   rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(cref.mttkrp(coords, vals, dims, A, n, nthreads=3), want,
                                   rtol=1e-12, atol=1e-12)


def test_unfolding_and_khatri_rao_by_hand():
    """X_(n) columns are mode-n fibers; KRP columns are Kronecker products."""
    X = np.arange(24, dtype=np.float64).reshape(2, 3, 4)
    U = ar.unfold(X, 1)
    assert U.shape == (3, 8)
    # column j of X_(1) is the fiber X[i0, :, i2] with j = i0*4 + i2
    np.testing.assert_array_equal(U[:, 1 * 4 + 2], X[1, :, 2])
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    B = np.array([[5.0, 6.0], [7.0, 8.0], [9.0, 10.0]])
    K = ar.khatri_rao([A, B])
    np.testing.assert_array_equal(K[:, 0], np.kron(A[:, 0], B[:, 0]))
    np.testing.assert_array_equal(K[:, 1], np.kron(A[:, 1], B[:, 1]))


def test_rank_one_closed_form():
    """X = a o b o c (dense, all cells stored): M_1(i,r) = a_i (b.B_r)(c.C_r)."""
    rng = np.random.default_rng(5)
    dims = (4, 5, 3)
    a, b, c = (rng.standard_normal(d) for d in dims)
    X = np.einsum("i,j,k->ijk", a, b, c)
    coords = np.stack(np.unravel_index(np.arange(X.size), dims)).astype(np.uint32)
    vals = X.reshape(-1).astype(np.float32)
    A = _factors(dims, 3, 1)
    got = ar.mttkrp(coords, vals, A, 0)
    v = vals.astype(np.float64).reshape(dims)  # the float32-rounded cells
    want = np.einsum("ijk,jr,kr->ir", v, A[1].astype(np.float64), A[2].astype(np.float64))
    np.testing.assert_allclose(got, want, rtol=1e-12)
    # and the factorised form with the exact rank-one tensor
    exact = np.outer(a, (b @ A[1].astype(np.float64)) * (c @ A[2].astype(np.float64)))
    np.testing.assert_allclose(got, exact, rtol=1e-5, atol=1e-6)


def test_all_ones_factors_give_slice_sums():
    dims = (30, 20, 10, 5)
    coords, vals = _random_tensor(dims, 2000, seed=2)
    A = [np.ones((d, 4), np.float32) for d in dims]
    for n in range(len(dims)):
        slice_sum = np.bincount(coords[n], weights=vals.astype(np.float64), minlength=dims[n])
        got = ar.mttkrp(coords, vals, A, n)
        for r in range(4):
            np.testing.assert_allclose(got[:, r], slice_sum, rtol=1e-12, atol=1e-12)
        got_c = cref.mttkrp(coords, vals, dims, A, n, nthreads=2)
        np.testing.assert_allclose(got_c[:, 0], slice_sum, rtol=1e-12, atol=1e-12)


def test_permutation_invariance_and_empty_rows():
    dims = (50, 40, 30)
    coords, vals = _random_tensor(dims, 400, seed=9)
    coords[0] = coords[0] % 25          # rows 25..49 of mode 0 stay empty
    A = _factors(dims, 5, 3)
    base = ar.mttkrp(coords, vals, A, 0)
    p = np.random.default_rng(1).permutation(400)
    perm = ar.mttkrp(coords[:, p], vals[p], A, 0)
    np.testing.assert_allclose(perm, base, rtol=1e-12, atol=1e-13)
    assert np.all(base[25:] == 0.0)


def test_rows_variant_matches_full():
    dims = (200, 50, 20)
    coords, vals = _random_tensor(dims, 5000, seed=4)
    A = _factors(dims, 8, 4)
    full = cref.mttkrp(coords, vals, dims, A, 0, nthreads=2)
    rows = np.array([0, 7, 199, 33], dtype=np.uint32)
    part = cref.mttkrp_rows(coords, vals, dims, A, 0, rows)
    np.testing.assert_array_equal(part, full[rows])


def test_c_linearize_matches_worked_example(worked_example):
    ex = worked_example
    rows = np.array(ex["nnz"], dtype=np.int64)
    coords = rows[:, :3].T.astype(np.uint32)
    keys = cref.linearize(coords, ex["dims"])[:, 0]
    srt = np.sort(keys)
    # the printed segments [2-20] and [25-51] bound the sorted keys
    assert (srt[0], srt[2], srt[3], srt[5]) == (2, 20, 25, 51)


def test_row_relative_error_metric():
    ref = np.array([[1.0, -2.0], [0.0, 0.0], [4.0, 4.0]])
    got = ref + np.array([[0.0, 2e-5], [0.0, 0.0], [0.0, -4e-5]])
    err, bad = ar.row_relative_error(got, ref)
    assert abs(err - 1e-5) < 1e-12 and bad == 0
    got[1, 0] = 1e-30
    assert ar.row_relative_error(got, ref)[1] == 1
