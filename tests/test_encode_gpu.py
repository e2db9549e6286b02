"""GPU encode parity through the C ABI: linear indices, ALTO order, partitions
and de-linearization are bit-exact against the oracle (Section III-A, IV-A)."""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _check(coords, vals, dims, L=None, host=False):
    import paper_2403_06348_gb300 as alto
    if host:
        t = alto.alto_encode(coords, vals, dims)
    else:
        t = gu.encode(coords, vals, dims)
    ref = ar.encode(coords, vals, dims)
    info = t.query()
    assert info.nbits == ref.plan.nbits
    assert info.key_words == ar.key_width_words(ref.plan.nbits)
    for n in range(len(dims)):
        mask = int(info.mask_lo[n]) | (int(info.mask_hi[n]) << 64)
        assert mask == ref.plan.masks[n]
    M = coords.shape[1]
    if M:
        keys, v = t.encoded()
        keys = keys.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(keys[:, 0], ref.lo)
        if info.key_words == 2:
            np.testing.assert_array_equal(keys[:, 1], ref.hi)
        np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), ref.vals.view(np.uint32))
        dc, dv = t.decode()
        np.testing.assert_array_equal(dc.cpu().numpy().view(np.uint32),
                                      ar.delinearize(ref.lo, ref.hi, ref.plan))
    norm = ar.tensor_norm_sq(coords, vals)
    assert abs(info.norm_sq - norm) <= 1e-9 * max(norm, 1.0)
    if L is not None:
        t.set_partitions(L)
    starts, iv = t.partition()
    Lg = len(starts) - 1
    rs, riv = ar.partition(ref, Lg)
    np.testing.assert_array_equal(starts, rs)
    np.testing.assert_array_equal(iv, riv)
    return t, ref


def test_worked_example(worked_example):
    ex = worked_example
    rows = np.array(ex["nnz"], dtype=np.int64)
    coords = rows[:, :3].T.astype(np.uint32)
    vals = rows[:, 3].astype(np.float32)
    t, ref = _check(coords, vals, ex["dims"], L=2)
    keys, _ = t.encoded()
    k = keys.cpu().numpy().view(np.uint64)[:, 0]
    starts, iv = t.partition()
    for l, seg in enumerate(ex["segment"]):
        a, b = int(starts[l]), int(starts[l + 1])
        assert (int(k[a]), int(k[b - 1])) == (seg[0], seg[1])
        np.testing.assert_array_equal(iv[l], np.array(seg[2:], dtype=np.uint32).reshape(3, 2))


@pytest.mark.parametrize("dims,M,seed", [
    ((1000, 800, 600), 100_000, 1),            # 30 bits, many sort tiles
    ((37, 1, 5000, 3), 3 * 4096 + 123, 2),     # a mode of length 1, ragged last tile
    ((1 << 20,) * 5, 50_000, 3),               # 100 bits: two-word positions
    ((2_000_000, 100_000, 10_000, 1000, 50), 20_000, 4),  # 68 bits
    ((7,), 1000, 5),                           # one mode
    ((2, 3), 1, 6),                            # a single nonzero
])
def test_random_tensors(dims, M, seed):
    coords, vals = gu.rand_tensor(dims, M, seed)
    _check(coords, vals, dims)


def test_duplicates_keep_input_order():
    dims = (4, 4, 4)
    rng = np.random.default_rng(0)
    coords = np.stack([rng.integers(0, 4, 20000) for _ in dims]).astype(np.uint32)
    vals = np.arange(20000, dtype=np.float32)
    _check(coords, vals, dims, L=7)


def test_empty_tensor():
    _check(np.zeros((3, 0), np.uint32), np.zeros(0, np.float32), (10, 20, 30), L=3)


def test_host_buffers():
    coords, vals = gu.rand_tensor((300, 200, 100), 5000, 9)
    _check(coords, vals, (300, 200, 100), host=True)


@pytest.mark.parametrize("L", [1, 13, 1000, 7000])
def test_partition_counts(L):
    coords, vals = gu.rand_tensor((500, 400, 300), 6000, 11)
    _check(coords, vals, (500, 400, 300), L=L)


def test_zipf_skewed_and_hot_rows():
    spec = synth.scaled(synth.ZIPF3D, 1_000_000)
    coords, vals = synth.generate(spec)
    t, ref = _check(coords, vals, spec.dims)
    for n, I in enumerate(spec.dims):
        hot = t.hot_rows(n)
        assert len(hot) == len(set(hot.tolist())) and (hot < I).all()
        if len(hot):
            counts = np.bincount(coords[n], minlength=I)
            assert hot[0] == int(np.argmax(counts))   # the Zipf head is found


def test_coordinate_out_of_range_is_reported():
    import paper_2403_06348_gb300 as alto
    coords, vals = gu.rand_tensor((10, 10), 100, 1)
    coords[1, 57] = 10
    with pytest.raises(alto.AltoError) as e:
        gu.encode(coords, vals, (10, 10))
    assert e.value.status == -5


def test_too_many_bits_unsupported():
    import paper_2403_06348_gb300 as alto
    with pytest.raises(alto.AltoError) as e:
        gu.encode(np.zeros((5, 4), np.uint32), np.ones(4, np.float32), (1 << 26,) * 5)
    assert e.value.status == -4


def test_device_inputs_of_the_wrong_dtype_are_refused():
    """CUDA tensors reach the library as raw pointers read as uint32 / float32;
    int64 coordinates or float64 values would be misread, so the binding
    refuses them before any call."""
    import torch
    import paper_2403_06348_gb300 as alto
    c = torch.zeros((3, 10), dtype=torch.int64, device="cuda")
    v = torch.ones(10, dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        alto.alto_encode(c, v, (4, 4, 4))
    with pytest.raises(TypeError):
        alto.alto_encode(c.to(torch.int32), v.double(), (4, 4, 4))
    t = alto.alto_encode(c.to(torch.int32), v, (4, 4, 4))
    assert t.nnz == 10
    t.free()


def _launched_passes(ref, nbits):
    """8-bit digits of the sort that are not the same for every nonzero: the
    passes the sort must launch (a constant digit leaves the order as it is)."""
    n = 0
    for p in range((nbits + 7) // 8):
        word, shift = divmod(8 * p, 64)
        k = ref.lo if word == 0 else ref.hi
        if len(np.unique((k >> np.uint64(shift)) & np.uint64(0xFF))) > 1:
            n += 1
    return n


@pytest.mark.parametrize("dims,limit,M,seed", [
    ((1 << 20,) * 3, 16, 50_000, 21),      # 60 bits, only the low 12 vary
    ((1 << 20,) * 5, 1024, 30_000, 22),    # 100 bits (two words), the high word constant
    ((1 << 22, 3, 1 << 18), 1 << 18, 20_000, 23),  # every digit varies
])
def test_constant_digits_are_skipped(dims, limit, M, seed):
    rng = np.random.default_rng(seed)
    coords = np.stack([rng.integers(0, min(d, limit), M) for d in dims]).astype(np.uint32)
    vals = (1.0 - rng.random(M)).astype(np.float32)
    t, ref = _check(coords, vals, dims)
    info = t.query()
    assert info.sort_passes == _launched_passes(ref, ref.plan.nbits)
    assert info.sort_passes < (ref.plan.nbits + 7) // 8 or limit >= 1 << 18
    assert info.encode_ms > 0 and 0 < info.sort_ms <= info.encode_ms


def test_every_digit_constant():
    """All nonzeros at one position: no pass runs, the values keep input order."""
    M = 9000
    coords = np.tile(np.array([[5], [700], [3]], np.uint32), (1, M))
    vals = np.arange(M, dtype=np.float32)
    t, _ = _check(coords, vals, (10, 1000, 4))
    assert t.query().sort_passes == 0


@pytest.mark.parametrize("M", [4095, 4096, 4097, 2 * 4096 + 1, 61 * 4096 - 7])
def test_sort_tile_edges(M):
    coords, vals = gu.rand_tensor((5000, 3000, 2000), M, M)
    _check(coords, vals, (5000, 3000, 2000))


@pytest.mark.parametrize("dims", [(1000, 800, 600), (1 << 20,) * 5])
def test_duplicates_across_passes_keep_input_order(dims):
    """500 distinct positions spread over every digit, drawn 200k times: equal
    positions must come out in input order through every pass and tile."""
    rng = np.random.default_rng(31)
    pool = np.stack([rng.integers(0, d, 500) for d in dims]).astype(np.uint32)
    pick = rng.integers(0, 500, 200_000)
    coords = np.ascontiguousarray(pool[:, pick])
    vals = np.arange(200_000, dtype=np.float32)
    _check(coords, vals, dims, L=11)


@pytest.mark.slow
def test_full_size_sort_bit_exact():
    """The 1e8-nonzero Zipf tensor of the bench (61-bit positions, eight sort
    passes, 24415 tiles per pass): every sorted position and value equals the
    oracle's stable order of its linear indices, bit for bit."""
    spec = synth.ZIPF3D
    coords, vals = synth.cached(spec)
    coords = np.asarray(coords)
    vals = np.asarray(vals)
    plan = ar.bit_plan(spec.dims)
    lo, _ = ar.linearize(coords, plan)
    perm = np.argsort(lo, kind="stable")
    t = gu.encode(coords, vals, spec.dims)
    keys, v = t.encoded()
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64)[:, 0], lo[perm])
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), vals[perm].view(np.uint32))
    assert t.query().sort_passes == 8
    t.free()
