"""alto_autotune: the measured per-mode plan (and segment count) stays set on
the handle, and MTTKRP under it still meets the fp32 bar on every mode."""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from oracle import cref
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


@pytest.mark.parametrize("name,nnz,R", [("COUNT4D", 1_000_000, 16), ("ZIPF3D", 1_000_000, 32),
                                         ("ZIPF5D", 300_000, 64)])
def test_autotuned_plans_keep_parity(name, nnz, R):
    spec = synth.scaled(getattr(synth, name), nnz)
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    A = gu.rand_factors(spec.dims, R, 9)
    Ad = gu.gpu_factors(A)
    rep = t.autotune(Ad, R, segments=True)
    N = len(spec.dims)
    assert rep["candidates"] >= 2 * N
    assert int(t.query().nparts) == rep["nparts"]
    for n in range(N):
        variant, cpl, hot = rep["plans"][n]
        # without the OUTPUT flag: the one-copy plans (line order, pull, in-tile)
        assert variant in (1, 2, 4, 5) and cpl in (4, 8)
        assert rep["ms"][n] > 0 and rep["default_ms"][n] > 0
        assert t.get_mode_plan(n, R)[:2] == (variant, cpl)
        got = t.mttkrp(n, Ad, R).cpu().numpy()
        ref = cref.mttkrp(coords, vals, spec.dims, A, n, nthreads=4)
        err, bad_zero = ar.row_relative_error(got, ref)
        assert bad_zero == 0 and err <= 1e-5, f"mode {n} plan {rep['plans'][n]}: {err:.3g}"
