"""CP-ALS batch (alto_batch_*): runs on different tensors advanced together.

Each run's fit trajectory must follow the fp64 oracle's (|dfit| <= 1e-4 per
iteration, the cpals_run bar) and match the same run done alone with
cpals_run, whether it ran alone in the batch or in a mix whose members join
and leave at different steps. A run with a singular V goes on through the
pseudo-inverse; a run with a non-finite V reports NOT_SPD; neither disturbs
the others.
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from oracle import cref
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

FIT_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _zipf(dims, nnz, seed):
    spec = synth.TensorSpec(f"b{seed}", tuple(dims), nnz, ("zipf:1.1",) * len(dims), "uniform01", 8,
                            seed=seed)
    return synth.generate(spec)


RUNS = [  # dims, nnz, R, iters
    ((300, 200, 100), 20_000, 8, 5),
    ((2_000, 500, 40, 12), 30_000, 16, 4),
    ((400, 300, 50, 20, 8), 25_000, 8, 3),
    ((5_000, 3_000, 200), 40_000, 32, 4),
    ((120, 90, 70), 3_000, 4, 6),
]


def _oracle_fits(coords, vals, dims, init, iters, tol=0.0):
    fn = lambda c, v, A, n: cref.mttkrp(c, v, dims, A, n, nthreads=4)  # noqa: E731
    return ar.cp_als(coords, vals, dims, init, iters, tol=tol, mttkrp_fn=fn)


class Run:
    def __init__(self, i, dims, nnz, R, iters, tol=0.0):
        self.dims, self.R, self.iters, self.tol = dims, R, iters, tol
        self.coords, self.vals = _zipf(dims, nnz, 300 + i)
        self.init = gu.rand_factors(dims, R, 400 + i)
        self.t = gu.encode(self.coords, self.vals, dims)

    def alone(self):
        A = gu.gpu_factors(self.init)
        lam, fits = self.t.cpals(self.R, self.iters, A, tol=self.tol)
        return A, lam, fits

    def fetch(self, batch, slot):
        import torch
        out = [torch.empty((d, self.R), device="cuda") for d in self.dims]
        lam = torch.empty(self.R, dtype=torch.float64, device="cuda")
        fits = torch.zeros(self.iters, dtype=torch.float64, device="cuda")
        done, status = batch.result(slot, out, lam, fits)
        batch.sync()
        return out, lam.cpu().numpy(), fits.cpu().numpy()[:done].tolist(), status


def _run_to_end(batch, slots, max_steps=1000):
    finished = set()
    for _ in range(max_steps):
        if finished >= set(slots):
            return finished
        batch.step(1)
        finished.update(batch.poll(wait=True))
    raise AssertionError("batch did not finish")


def test_batch_matches_oracle_and_alone():
    import paper_2403_06348_gb300 as alto
    runs = [Run(i, *c) for i, c in enumerate(RUNS)]
    batch = alto.Batch(max_slots=16)
    slots = [batch.add(r.t, r.R, r.iters, gu.gpu_factors(r.init)) for r in runs]
    _run_to_end(batch, slots)
    for r, s in zip(runs, slots):
        A, lam, fits, status = r.fetch(batch, s)
        assert status == 0
        ref = _oracle_fits(r.coords, r.vals, r.dims, r.init, r.iters)
        np.testing.assert_allclose(fits, ref.fits, atol=FIT_TOL)
        _, lam1, fits1 = r.alone()
        np.testing.assert_allclose(fits, fits1, atol=FIT_TOL)
        np.testing.assert_allclose(np.sort(lam), np.sort(lam1), rtol=1e-2)
        for a in A:  # normalised columns
            np.testing.assert_allclose(a.norm(dim=0).cpu().numpy(), 1.0, rtol=1e-4)
        batch.remove(s)
    assert batch.info().active == 0
    batch.free()


def test_runs_join_and_leave_between_steps():
    """Continuous batching: runs admitted while others are mid-way, slots
    reused after removal; every result equals the run done alone."""
    import paper_2403_06348_gb300 as alto
    runs = [Run(10 + i, *c) for i, c in enumerate(RUNS)]
    alone = [r.alone()[2] for r in runs]
    batch = alto.Batch(max_slots=3)  # fewer slots than runs: slots are reused
    pending = list(range(len(runs)))
    live = {}
    results = {}
    steps = 0
    while pending or live:
        while pending and len(live) < 3 and (steps % 2 == 0 or not live):
            i = pending.pop(0)
            live[batch.add(runs[i].t, runs[i].R, runs[i].iters, gu.gpu_factors(runs[i].init))] = i
        batch.step(1)
        steps += 1
        for s in batch.poll(wait=True):
            i = live.pop(s)
            _, _, fits, status = runs[i].fetch(batch, s)
            assert status == 0
            results[i] = fits
            batch.remove(s)
        assert steps < 500
    for i in range(len(runs)):
        np.testing.assert_allclose(results[i], alone[i], atol=FIT_TOL)
    batch.free()


def test_tol_stop_pinv_and_not_spd_in_the_mix():
    import paper_2403_06348_gb300 as alto
    good = Run(20, (300, 200, 100), 20_000, 8, 40, tol=1e-3)
    sing = Run(21, (60, 50, 40), 3_000, 4, 5)
    for a in sing.init:
        a[:, 1] = 0.0  # a zero column in every factor: V is singular (pseudo-inverse)
    bad = Run(23, (60, 50, 40), 3_000, 4, 5)
    bad.init[1][7, 2] = np.inf  # a non-finite V: the run ends with NOT_SPD
    plain = Run(22, (500, 400, 30), 15_000, 16, 4)
    batch = alto.Batch(max_slots=8)
    sg = batch.add(good.t, good.R, good.iters, gu.gpu_factors(good.init), tol=good.tol)
    ss = batch.add(sing.t, sing.R, sing.iters, gu.gpu_factors(sing.init))
    sb = batch.add(bad.t, bad.R, bad.iters, gu.gpu_factors(bad.init))
    sp = batch.add(plain.t, plain.R, plain.iters, gu.gpu_factors(plain.init))
    _run_to_end(batch, [sg, ss, sb, sp])
    _, _, fits_g, st_g = good.fetch(batch, sg)
    _, _, fits_s, st_s = sing.fetch(batch, ss)
    _, _, _, st_b = bad.fetch(batch, sb)
    _, _, fits_p, st_p = plain.fetch(batch, sp)
    assert st_b == -6 and st_g == 0 and st_p == 0 and st_s == 0
    ref_s = _oracle_fits(sing.coords, sing.vals, sing.dims, sing.init, sing.iters)
    np.testing.assert_allclose(fits_s, ref_s.fits, atol=FIT_TOL)
    _, _, alone_g = good.alone()
    assert 1 < len(fits_g) < good.iters and len(fits_g) == len(alone_g)
    np.testing.assert_allclose(fits_g, alone_g, atol=FIT_TOL)
    np.testing.assert_allclose(fits_p, plain.alone()[2], atol=FIT_TOL)
    batch.free()


def test_host_factors_in_and_out():
    import paper_2403_06348_gb300 as alto
    r = Run(30, (200, 150, 100), 10_000, 8, 3)
    batch = alto.Batch(max_slots=2)
    s = batch.add(r.t, r.R, r.iters, [a.copy() for a in r.init])  # host factors copied in
    _run_to_end(batch, [s])
    out = [np.empty((d, r.R), dtype=np.float32) for d in r.dims]
    lam = np.empty(r.R)
    fits = np.zeros(r.iters)
    done, status = batch.result(s, out, lam, fits)
    batch.sync()
    assert status == 0 and done == r.iters
    A1, lam1, fits1 = r.alone()
    np.testing.assert_allclose(fits, fits1, atol=FIT_TOL)
    ref = _oracle_fits(r.coords, r.vals, r.dims, r.init, r.iters)
    np.testing.assert_allclose(fits, ref.fits, atol=FIT_TOL)
    batch.free()


def test_batch_bad_arguments():
    import torch
    import paper_2403_06348_gb300 as alto
    batch = alto.Batch(max_slots=1)
    r = Run(40, (50, 40, 30), 2_000, 8, 2)
    A = gu.gpu_factors(r.init)
    with pytest.raises(alto.AltoError) as e:
        batch.add(r.t, 12, 2, A)
    assert e.value.status == -4
    s = batch.add(r.t, 8, 2, A)
    with pytest.raises(alto.AltoError) as e:  # one slot only
        batch.add(r.t, 8, 2, A)
    assert e.value.status == -4
    with pytest.raises(alto.AltoError):       # not finished yet
        batch.result(s, [torch.empty((d, 8), device="cuda") for d in r.dims])
    batch.remove(s)
    with pytest.raises(alto.AltoError):
        batch.remove(s)
    batch.free()
