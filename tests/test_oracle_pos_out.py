"""Pins for the oracle's output-oriented traversal (Alg. 4): the stored order
pos_out and the traversal that walks it.

pos_out is checked against brute force over every permutation of small
segments, against the mode intervals the paper prints for its worked example
(the first and last nonzero of a segment in pos_out order sit at T^s and
T^e), and against the permutation and ordering invariants on larger random
tensors. The traversal is checked against the dense unfolding times the
Khatri-Rao product, its update count against the number of distinct rows per
segment, and its boundary count against the rows that segments share.
"""
import itertools

import numpy as np
import pytest

from oracle import alto_ref as ar


def _random_tensor(dims, M, seed):
    rng = np.random.default_rng(seed)
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    vals = rng.standard_normal(M).astype(np.float32)
    return coords, vals


def _factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((d, R)).astype(np.float32) for d in dims]


@pytest.mark.parametrize("dims,M,L", [((4, 3, 2), 7, 1), ((4, 3, 2), 7, 2), ((3, 3), 6, 3),
                                       ((2, 5, 2, 3), 6, 2), ((6,), 5, 2)])
def test_pos_out_brute_force(dims, M, L):
    """The only ordering of each segment whose output coordinates never
    decrease and whose equal coordinates keep line order."""
    coords, vals = _random_tensor(dims, M, seed=M * 10 + L)
    t = ar.encode(coords, vals, dims)
    C = ar.delinearize(t.lo, t.hi, t.plan)
    starts = ar.segment_starts(M, L)
    for n in range(len(dims)):
        got = ar.pos_out(t, L, n)
        for l in range(L):
            a, b = int(starts[l]), int(starts[l + 1])
            ok = []
            for perm in itertools.permutations(range(a, b)):
                rows = [int(C[n, x]) for x in perm]
                if all(rows[k] < rows[k + 1] or (rows[k] == rows[k + 1] and perm[k] < perm[k + 1])
                       for k in range(len(perm) - 1)):
                    ok.append(perm)
            assert len(ok) == 1
            assert tuple(got[a:b].tolist()) == ok[0]


def test_pos_out_ends_at_printed_intervals(worked_example):
    """Section IV-A prints the two segments of the example tensor with mode
    intervals {[0-3],[0-3],[0-1]} and {[1-3],[2-6],[0-1]}: in pos_out order of
    mode n a segment starts at T^s_n and ends at T^e_n."""
    ex = worked_example
    rows = np.array(ex["nnz"], dtype=np.int64)
    coords = rows[:, :3].T.astype(np.uint32)
    vals = rows[:, 3].astype(np.float32)
    t = ar.encode(coords, vals, ex["dims"])
    C = ar.delinearize(t.lo, t.hi, t.plan)
    starts = ar.segment_starts(t.nnz, 2)
    for l, seg in enumerate(ex["segment"]):
        a, b = int(starts[l]), int(starts[l + 1])
        for n in range(3):
            po = ar.pos_out(t, 2, n)
            lo, hi = seg[2 + 2 * n], seg[3 + 2 * n]
            assert (int(C[n, po[a]]), int(C[n, po[b - 1]])) == (lo, hi)


@pytest.mark.parametrize("dims,M,L", [((50, 40, 7), 3000, 13), ((9, 300, 4, 20), 2500, 1),
                                       ((1000, 3), 999, 64), ((17, 5, 3, 2, 11), 1200, 7),
                                       ((30, 30, 30), 50, 200)])
def test_pos_out_invariants(dims, M, L):
    coords, vals = _random_tensor(dims, M, seed=M + L)
    t = ar.encode(coords, vals, dims)
    C = ar.delinearize(t.lo, t.hi, t.plan)
    starts = ar.segment_starts(M, L)
    for n in range(len(dims)):
        po = ar.pos_out(t, L, n)
        for l in range(L):
            a, b = int(starts[l]), int(starts[l + 1])
            seg = po[a:b]
            np.testing.assert_array_equal(np.sort(seg), np.arange(a, b))
            r = C[n, seg].astype(np.int64)
            assert np.all(np.diff(r) >= 0)
            same = np.diff(r) == 0
            assert np.all(np.diff(seg)[same] > 0)
    # one segment holding everything: pos_out is a stable sort of the whole line
    po = ar.pos_out(t, 1, 0)
    want = sorted(range(M), key=lambda x: (int(C[0, x]), x))
    np.testing.assert_array_equal(po, want)


@pytest.mark.parametrize("dims,M,L,R", [((6, 5, 4), 80, 3, 3), ((4, 8, 2), 6, 2, 2),
                                         ((5, 3, 4, 6), 150, 5, 4), ((3, 2, 2, 3, 2), 60, 4, 2),
                                         ((40, 3), 100, 1, 3)])
def test_output_oriented_traversal(dims, M, L, R):
    coords, vals = _random_tensor(dims, M, seed=7 * M + L)
    A = _factors(dims, R, seed=R + L)
    X = ar.to_dense(coords, vals, dims)
    t = ar.encode(coords, vals, dims)
    C = ar.delinearize(t.lo, t.hi, t.plan)
    starts = ar.segment_starts(M, L)
    for n in range(len(dims)):
        got, updates, boundary = ar.mttkrp_output_oriented(t, A, n, L)
        np.testing.assert_allclose(got, ar.mttkrp_dense(X, A, n), rtol=1e-12, atol=1e-12)
        segs = [set(C[n, int(starts[l]):int(starts[l + 1])].tolist()) for l in range(L)]
        assert updates == sum(len(s) for s in segs)
        shared = sum(1 for l in range(L) for i in segs[l]
                     if any(i in segs[k] for k in range(L) if k != l))
        assert boundary == shared
        if L == 1:
            assert boundary == 0
