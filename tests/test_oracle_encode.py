"""Pins for the oracle's encode: bit plan, linearization, ordering, partitions.

Each test ties oracle.alto_ref to something other than itself: numbers printed
in the paper (tests/golden/worked_example.txt), brute force over every point
of small boxes, and invariants that follow from the definitions.
"""
import itertools

import numpy as np
import pytest

from oracle import alto_ref as ar


def _example_arrays(ex):
    rows = np.array(ex["nnz"], dtype=np.int64)
    coords = rows[:, :3].T.astype(np.uint32)
    vals = rows[:, 3].astype(np.float32)
    return coords, vals


def test_worked_example_bits_and_line(worked_example):
    ex = worked_example
    plan = ar.bit_plan(ex["dims"])
    assert plan.nbits == ex["index_bits"]
    assert 1 << plan.nbits == ex["line_length"]


def test_worked_example_prefix_subspaces(worked_example):
    """Section III-A: the prefix [0, P) of the line is exactly a sub-box."""
    ex = worked_example
    plan = ar.bit_plan(ex["dims"])
    for P, a, b, c in ex["prefix"]:
        inside = {pt for pt in itertools.product(*map(range, ex["dims"]))
                  if ar.linearize_one(pt, plan) < P}
        assert inside == set(itertools.product(range(a), range(b), range(c)))


def test_worked_example_segments(worked_example):
    """Section IV-A: two balanced segments and their mode intervals."""
    ex = worked_example
    coords, vals = _example_arrays(ex)
    t = ar.encode(coords, vals, ex["dims"])
    L = len(ex["segment"])
    starts, iv = ar.partition(t, L)
    keys = t.lo.astype(np.int64)
    for l, seg in enumerate(ex["segment"]):
        a, b = int(starts[l]), int(starts[l + 1])
        assert (keys[a], keys[b - 1]) == (seg[0], seg[1])
        want = np.array(seg[2:], dtype=np.uint32).reshape(3, 2)
        np.testing.assert_array_equal(iv[l], want)
    # the two segments hold the same number of nonzeros
    assert int(starts[1] - starts[0]) == int(starts[2] - starts[1])


def test_worked_example_storage(worked_example):
    ex = worked_example
    dims = ex["dims"]
    assert ar.coo_over_alto(dims, 8) == ex["coo_over_alto_wb8"]
    M = len(ex["nnz"])
    # Eq. 3 vs Eq. 1 expressed as line lengths 2^(bits per nonzero)
    sfc = ar.storage_bits_sfc(dims, M) // M
    alto = ar.storage_bits_alto(dims, M) // M
    assert 2 ** (sfc - alto) == ex["sfc_line_factor"]


def test_eq1_eq2_closed_forms():
    # Eq. 1 with powers of two: log2 exactly
    assert ar.storage_bits_alto((1 << 10, 1 << 7, 4), 5) == 5 * (10 + 7 + 2)
    # Eq. 2 is >= 1 always and equals N when every mode fits one word and the
    # sum fits one word too
    assert ar.coo_over_alto((3, 5, 7, 9), 64) == 4
    for dims in [(10_000_000, 2_000_000, 50_000), (1_000_000, 500_000, 200, 24), (2, 2)]:
        assert ar.coo_over_alto(dims, 64) >= 1
        assert ar.coo_over_alto(dims, 8) >= 1


def test_mode_bits():
    assert [ar.mode_bits(i) for i in (1, 2, 3, 4, 5, 8, 9, 1 << 20, (1 << 20) + 1)] == \
        [0, 1, 2, 2, 3, 3, 4, 20, 21]


@pytest.mark.parametrize("dims", [(4, 8, 2), (2, 2, 2), (16, 4), (8, 1, 4), (2, 4, 8, 2)])
def test_bijection_on_power_of_two_boxes(dims):
    """With power-of-two dims the line is exactly the box: a bijection."""
    plan = ar.bit_plan(dims)
    keys = [ar.linearize_one(pt, plan) for pt in itertools.product(*map(range, dims))]
    assert sorted(keys) == list(range(1 << plan.nbits))
    for pt in itertools.product(*map(range, dims)):
        assert ar.delinearize_one(ar.linearize_one(pt, plan), plan) == pt


@pytest.mark.parametrize("dims", [(3, 5, 7), (6, 1, 9), (100, 3)])
def test_injective_on_ragged_boxes(dims):
    plan = ar.bit_plan(dims)
    keys = [ar.linearize_one(pt, plan) for pt in itertools.product(*map(range, dims))]
    assert len(set(keys)) == len(keys)
    assert max(keys) < (1 << plan.nbits)


def test_shortest_mode_at_lowest_bit():
    """Section III-A: inside a group the shortest mode gets the lowest bit; a
    tie in length keeps the lower mode index lower."""
    plan = ar.bit_plan((8, 2, 4))
    # group 0: mode 1 (len 2), mode 2 (len 4), mode 0 (len 8)
    assert plan.positions[1][0] == 0 and plan.positions[2][0] == 1 and plan.positions[0][0] == 2
    plan = ar.bit_plan((4, 4))
    assert plan.positions[0] == (0, 2) and plan.positions[1] == (1, 3)


@pytest.mark.parametrize("dims,M", [((1000, 800, 600), 5000), ((2_000_000, 100_000, 10_000, 1000, 50), 4000),
                                     ((1 << 20,) * 5, 3000), ((5, 1, 3), 50)])
def test_vectorised_round_trip(dims, M):
    rng = np.random.default_rng(7)
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    plan = ar.bit_plan(dims)
    lo, hi = ar.linearize(coords, plan)
    np.testing.assert_array_equal(ar.delinearize(lo, hi, plan), coords)
    # the vectorised gather agrees with the bit-by-bit Python-int gather
    for x in range(0, M, max(1, M // 50)):
        k = ar.linearize_one(tuple(int(c) for c in coords[:, x]), plan)
        assert k == int(lo[x]) | (int(hi[x]) << 64)
    if plan.nbits <= 64:
        assert not hi.any()


def test_ordering_is_stable_and_sorted():
    dims = (16, 16, 16)
    rng = np.random.default_rng(3)
    M = 3000
    coords = np.stack([rng.integers(0, 4, M) for _ in dims]).astype(np.uint32)  # many duplicates
    vals = np.arange(M, dtype=np.float32)
    t = ar.encode(coords, vals, dims)
    k = [int(a) | (int(b) << 64) for a, b in zip(t.lo, t.hi)]
    assert all(k[i] <= k[i + 1] for i in range(M - 1))
    # equal keys keep input order: values (= input index) increase inside each run
    for i in range(M - 1):
        if k[i] == k[i + 1]:
            assert t.vals[i] < t.vals[i + 1]
    assert sorted(t.perm.tolist()) == list(range(M))


@pytest.mark.parametrize("M,L", [(1000, 7), (10, 3), (5, 8), (0, 2), (4096, 4096)])
def test_partition_balanced_and_tight(M, L):
    dims = (50, 20, 30)
    rng = np.random.default_rng(11)
    coords = np.stack([rng.integers(0, d, M) for d in dims]).astype(np.uint32)
    t = ar.encode(coords, np.ones(M, np.float32), dims)
    starts, iv = ar.partition(t, L)
    sizes = np.diff(starts.astype(np.int64))
    assert sizes.sum() == M and sizes.max() - sizes.min() <= 1
    dec = ar.delinearize(t.lo, t.hi, t.plan)
    for l in range(L):
        a, b = int(starts[l]), int(starts[l + 1])
        for n in range(3):
            if b > a:
                seg = dec[n, a:b]
                assert iv[l, n, 0] == seg.min() and iv[l, n, 1] == seg.max()
            else:
                assert iv[l, n, 0] == ar.EMPTY_LO and iv[l, n, 1] == 0


def test_reuse_classes():
    """Section V-A: high above 8, medium 5..8, limited below 5."""
    assert [ar.reuse_class(r) for r in (100, 8.5, 8, 5, 4.9, 1)] == \
        ["high", "high", "medium", "medium", "limited", "limited"]
    assert ar.fiber_reuse(200, (10, 40)) == [20.0, 5.0]


def test_too_many_bits_rejected():
    with pytest.raises(ValueError):
        ar.encode(np.zeros((5, 1), np.uint32), np.ones(1, np.float32), (1 << 26,) * 5)
