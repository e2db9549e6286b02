"""The serving loop (paper_2403_06348_gb300.serve.Server): requests admitted
while others run give the same CP-ALS result as each request solved alone with
cpals_run (fits within 1e-4 per iteration), under a roomy and a tight device
memory budget."""
import numpy as np
import pytest

import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _requests(n, seed):
    pool, reqs = synth.request_pool_stream(count=n, pool=n, seed=seed, nnz_range=(2_000, 60_000),
                                           dim_range=(50, 20_000), iters=4)
    data = {p.rid: synth.request_tensor(p) for p in pool}
    return [(r, data[r.rid]) for r in reqs]


def _alone(req, coords, vals):
    import paper_2403_06348_gb300 as alto
    from paper_2403_06348_gb300 import serve
    t = alto.alto_encode(coords, vals, req.dims)
    A = serve.device_factors(req.dims, req.rank, req.seed % (1 << 27))
    try:
        lam, fits = t.cpals(req.rank, req.iters, A)
    finally:
        t.free()
    return fits


@pytest.mark.parametrize("budget", [100e9, 1.0])   # 1 byte: one request at a time
def test_served_results_equal_alone(budget):
    from paper_2403_06348_gb300 import serve
    reqs = _requests(12, 77)
    srv = serve.Server(budget_bytes=budget, max_slots=8)
    futs = [srv.submit(c, v, r.dims, r.rank, r.iters, seed=r.seed % (1 << 27)) for r, (c, v) in reqs]
    results = [f.result(timeout=300) for f in futs]
    srv.close()
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["errors"] == 0
    assert 0.0 < st["p50_s"] <= st["p99_s"]
    for (r, (c, v)), res in zip(reqs, results):
        assert res.status == 0 and res.iters_done == r.iters
        np.testing.assert_allclose(res.fits, _alone(r, c, v), atol=1e-4)
        for a, d in zip(res.factors, r.dims):
            assert a.shape == (d, r.rank)
            norms = np.linalg.norm(a, axis=0)
            np.testing.assert_allclose(norms[res.lam > 0], 1.0, rtol=1e-4)


def test_fcfs_reference_runs_the_same_requests():
    from paper_2403_06348_gb300 import serve
    import time
    reqs = _requests(4, 78)
    items = [(0.0, c, v, r.dims, r.rank, r.iters, None, r.seed % (1 << 27)) for r, (c, v) in reqs]
    st = serve.run_fcfs(items, time.perf_counter())
    assert st["completed"] == 4 and st["not_spd"] == 0 and st["p99_s"] > 0
