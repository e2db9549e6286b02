"""CP-APR on the GPU (Phi kernel of Alg. 5, MU loop of Alg. 2) through the C
ABI against the fp64 oracle in oracle/apr_ref.py.

Phi: max row-relative error <= 1e-5 (the MTTKRP bar) for both conflict
resolutions (ATOMIC with hot rows, PULL) and both ways of forming the
Khatri-Rao rows (on the fly, precomputed). The MU loop: the objective after
every outer iteration within 1e-5 (relative) of the oracle's while the inner
step counts agree, the rank-1 closed form, the fixed point of an exact model,
and PRE equal to OTF.
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from oracle import apr_ref as apr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def _count_tensor(dims, nnz, seed):
    spec = synth.TensorSpec(f"apr{seed}", tuple(dims), nnz,
                            ("zipf:1.2",) * 2 + ("uniform",) * (len(dims) - 2), "poisson3p1", 8,
                            seed=seed)
    return synth.generate(spec)


def _pos(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [(0.1 + rng.random((d, R))).astype(np.float32) for d in dims]


@pytest.mark.parametrize("variant", [1, 2, 3])       # ATOMIC, PULL, OUTPUT
@pytest.mark.parametrize("pre", [False, True])
@pytest.mark.parametrize("R", [4, 16, 32])
def test_phi_matches_oracle(variant, pre, R):
    dims = (300, 200, 24)
    coords, vals = _count_tensor(dims, 40_000, 3)
    t = gu.encode(coords, vals, dims)
    A = _pos(dims, R, 4)
    Ad = gu.gpu_factors(A)
    for n in range(3):
        t.set_mode_plan(n, variant, 4)
        assert t.get_mode_plan(n, R)[0] == variant
        B = _pos([dims[n]], R, 5 + n)[0]
        got = t.phi(n, Ad, gu.to_dev(B), R, pre=pre).cpu().numpy()
        ref = apr.phi(coords, vals, dims, A, B, n)
        err, bad_zero = ar.row_relative_error(got, ref)
        assert bad_zero == 0, f"mode {n}: rows without nonzeros are not 0"
        assert err <= 1e-5, f"mode {n} R {R} pre {pre}: {err:.3g}"


@pytest.mark.parametrize("variant", [1, 3])          # ATOMIC, OUTPUT
def test_phi_four_and_five_modes_wide_keys(variant):
    for dims in [(500, 400, 30, 12), (2_000_000, 100_000, 10_000, 1000, 50),
                 (40, 30, 20, 10, 8, 6)]:
        coords, vals = _count_tensor(dims, 30_000, 6)
        t = gu.encode(coords, vals, dims)
        A = _pos(dims, 16, 7)
        Ad = gu.gpu_factors(A)
        for n in range(len(dims)):
            t.set_mode_plan(n, variant, 4)
            B = _pos([dims[n]], 16, 8)[0]
            for pre in (False, True):
                got = t.phi(n, Ad, gu.to_dev(B), 16, pre=pre).cpu().numpy()
                err, bad = ar.row_relative_error(got, apr.phi(coords, vals, dims, A, B, n))
                assert bad == 0 and err <= 1e-5, f"{dims} mode {n} pre {pre}: {err:.3g}"


def test_cpapr_follows_the_oracle():
    dims, R = (200, 150, 24), 8
    coords, vals = _count_tensor(dims, 20_000, 9)
    init = _pos(dims, R, 10)
    ref = apr.cp_apr_mu(coords, vals, dims, init, k_max=6)
    t = gu.encode(coords, vals, dims)
    A = gu.gpu_factors(init)
    got = t.cpapr(R, A, k_max=6)
    k = min(got["outer_done"], ref.outer_done)
    # the trajectories are comparable while the KKT tests took the same steps
    same = 0
    while same < k and got["inner"][same] == ref.inner[same]:
        same += 1
    assert same >= 2, (got["inner"], ref.inner)
    np.testing.assert_allclose(got["objective"][:same], ref.objective[:same], rtol=1e-5)
    f = np.array(got["objective"])
    assert np.all(np.diff(f) <= 1e-6 * np.abs(f[:-1])), "objective increased"
    for a in A:
        np.testing.assert_allclose(a.sum(dim=0).cpu().numpy(), 1.0, rtol=1e-4)


def test_cpapr_rank_one_marginals():
    dims = (120, 90, 30)
    coords, vals = _count_tensor(dims, 15_000, 11)
    t = gu.encode(coords, vals, dims)
    # R = 1 is not a library rank; R = 4 with four identical columns follows
    # the rank-1 iteration in every column and ends at the marginals
    A4 = [a[:, :1].repeat(1, 4).contiguous() for a in gu.gpu_factors(_pos(dims, 4, 12))]
    got = t.cpapr(4, A4, k_max=10)
    total = float(vals.astype(np.float64).sum())
    np.testing.assert_allclose(got["lam"].sum(), total, rtol=1e-5)
    for n in range(3):
        marg = np.bincount(coords[n], weights=vals.astype(np.float64), minlength=dims[n]) / total
        for r in range(4):
            np.testing.assert_allclose(A4[n][:, r].double().cpu().numpy(), marg, rtol=1e-4, atol=1e-8)


def test_cpapr_exact_model_is_a_fixed_point():
    dims, R = (12, 10, 8), 4
    lam, A = apr.normalize([a.astype(np.float64) for a in _pos(dims, R, 13)])
    X = ar.reconstruct_dense(lam, A)
    coords = np.stack(np.nonzero(X > -1)).astype(np.uint32)
    vals = X[tuple(coords)].astype(np.float32)
    t = gu.encode(coords, vals, dims)
    init = [A[0] * lam[None, :]] + A[1:]
    Ad = gu.gpu_factors([a.astype(np.float32) for a in init])
    got = t.cpapr(R, Ad, k_max=5)
    assert got["converged"] and got["outer_done"] == 1 and got["inner_steps_total"] == 0


def test_cpapr_output_traversal_follows_the_oracle():
    """Every mode on the stored output-oriented order (OUTPUT), PRE and OTF."""
    import paper_2403_06348_gb300 as alto
    dims, R = (200, 150, 24), 8
    coords, vals = _count_tensor(dims, 20_000, 9)
    init = _pos(dims, R, 10)
    ref = apr.cp_apr_mu(coords, vals, dims, init, k_max=6)
    for variant in (alto.APR_OTF, alto.APR_PRE):
        t = gu.encode(coords, vals, dims)
        for n in range(3):
            t.set_mode_plan(n, alto.VARIANT_OUTPUT, 4)
        got = t.cpapr(R, gu.gpu_factors(init), k_max=6, variant=variant)
        k = min(got["outer_done"], ref.outer_done)
        same = 0
        while same < k and got["inner"][same] == ref.inner[same]:
            same += 1
        assert same >= 2, (got["inner"], ref.inner)
        np.testing.assert_allclose(got["objective"][:same], ref.objective[:same], rtol=1e-5)


def test_cpapr_pre_equals_otf_and_host_factors():
    dims, R = (400, 300, 24, 8), 16
    coords, vals = _count_tensor(dims, 30_000, 14)
    t = gu.encode(coords, vals, dims)
    init = _pos(dims, R, 15)
    import paper_2403_06348_gb300 as alto
    A1 = gu.gpu_factors(init)
    otf = t.cpapr(R, A1, k_max=4, variant=alto.APR_OTF)
    A2 = gu.gpu_factors(init)
    pre = t.cpapr(R, A2, k_max=4, variant=alto.APR_PRE)
    assert pre["pre_modes"] == 4 and otf["pre_modes"] == 0
    assert pre["inner"] == otf["inner"]
    np.testing.assert_allclose(pre["objective"], otf["objective"], rtol=1e-5)
    Ah = [a.copy() for a in init]
    host = t.cpapr(R, Ah, k_max=4, variant=alto.APR_OTF)
    np.testing.assert_allclose(host["objective"], otf["objective"], rtol=1e-5)
    for a, b in zip(Ah, A1):
        np.testing.assert_allclose(a, b.cpu().numpy(), rtol=1e-3, atol=1e-6)


def test_cpapr_bad_arguments():
    import torch
    import paper_2403_06348_gb300 as alto
    coords, vals = _count_tensor((20, 20, 20), 500, 16)
    t = gu.encode(coords, vals, (20, 20, 20))
    A = gu.gpu_factors(_pos((20, 20, 20), 8, 17))
    with pytest.raises(alto.AltoError):
        t.cpapr(12, A, k_max=2)
    with pytest.raises(alto.AltoError):
        t.cpapr(8, A, k_max=0)
    with pytest.raises(alto.AltoError):
        t.cpapr(8, A, k_max=2, tau=0.0)
