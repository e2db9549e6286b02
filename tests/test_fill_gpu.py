"""alto_fill_uniform against SplitMix64 written out here in numpy (wrapping
uint64 arithmetic): every element bit-exact."""
import numpy as np
import pytest

from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def splitmix64_uniform(seed, n):
    with np.errstate(over="ignore"):
        x = (np.uint64(seed) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)


@pytest.mark.parametrize("seed,n", [(0, 1), (1, 1000), (12345, 100_003), (2**32 - 1, 4097)])
def test_fill_uniform_bit_exact(seed, n):
    import torch
    import paper_2403_06348_gb300 as alto
    gu.ensure_built()
    x = torch.full((n,), -1.0, device="cuda")
    alto.alto_fill_uniform(x, seed)
    got = x.cpu().numpy()
    np.testing.assert_array_equal(got, splitmix64_uniform(seed, n))
    assert got.min() >= 0.0 and got.max() < 1.0


def test_fill_uniform_rejects_bad_seed():
    import torch
    import paper_2403_06348_gb300 as alto
    gu.ensure_built()
    with pytest.raises(alto.AltoError):
        alto.alto_fill_uniform(torch.empty(4, device="cuda"), 2**32)
