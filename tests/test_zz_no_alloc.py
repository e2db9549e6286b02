"""alto_mttkrp_noalloc: the MTTKRP entry point for callers that cannot have
the library allocate device memory while they run.

Its partials live in a fixed device array inside the library instead of a
buffer the library allocates, so its results must equal those of the regular
entry point (same tolerance as every fp32 MTTKRP test: 1e-5 row-relative),
call after call: the array keeps the previous call's contents. This file is
named to be collected last.
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


def test_noalloc_matches_regular_entry_point_on_two_calls():
    import torch
    import paper_2403_06348_gb300 as alto
    spec = synth.scaled(synth.COUNT4D, 400_000)   # count tensor: 200- and 24-row modes
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    R = 16
    A = gu.gpu_factors(gu.rand_factors(spec.dims, R, 3))
    for mode in (2, 3):
        t.set_mode_plan(mode, alto.VARIANT_PULL)
        ref = t.mttkrp(mode, A, R).cpu().numpy()      # regular entry point; builds the pull lists
        for call in range(2):
            out = torch.full((spec.dims[mode], R), float("nan"), device="cuda")
            alto.alto_mttkrp_noalloc(t, mode, A, R, out)
            got = out.cpu().numpy()
            err, bad_zero = ar.row_relative_error(got, ref)
            assert bad_zero == 0 and err <= TOL_F32, (mode, call, err)


def test_noalloc_rejects_what_it_cannot_do():
    import torch
    import paper_2403_06348_gb300 as alto
    spec = synth.scaled(synth.COUNT4D, 400_000)
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    R = 64
    A = gu.gpu_factors(gu.rand_factors(spec.dims, R, 4))
    out = torch.empty((spec.dims[2], R), device="cuda")
    # lists not built yet for this mode: refused, nothing launched
    with pytest.raises(alto.AltoError) as e:
        alto.alto_mttkrp_noalloc(t, 2, A, R, out)
    assert e.value.status == -1
    # more partial rows than the fixed scratch holds: refused with the sizes
    t.set_partitions(200_000)                           # 200 rows x 200k segments x 64 > 8 Mi
    t.set_mode_plan(2, alto.VARIANT_PULL)
    t.mttkrp(2, A, R, out=out)
    with pytest.raises(alto.AltoError) as e:
        alto.alto_mttkrp_noalloc(t, 2, A, R, out)
    assert e.value.status == -4 and "scratch" in str(e.value)
