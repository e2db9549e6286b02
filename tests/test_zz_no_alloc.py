"""alto_mttkrp_noalloc: the MTTKRP entry point for callers that cannot have
the library allocate device memory while they run.

Its partials live in a fixed device array inside the library instead of a
buffer the library allocates. Its results must match the fp64 oracle within
the bar of every MTTKRP test (1e-5 row-relative for fp32 factors, 1e-2 for
bf16 factors against the oracle on the original fp32 factors), and the
regular entry point within the same bar, call after call: the array keeps the
previous call's contents. This file is named to be collected last.
"""
import numpy as np
import pytest

import synth
from oracle import alto_ref as ar
from oracle import cref
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    gu.ensure_built()


@pytest.mark.parametrize("bf16", [False, True])
def test_noalloc_matches_oracle_and_regular_entry_point_on_two_calls(bf16):
    import torch
    import paper_2403_06348_gb300 as alto
    spec = synth.scaled(synth.COUNT4D, 400_000)   # count tensor: 200- and 24-row modes
    coords, vals = synth.generate(spec)
    t = gu.encode(coords, vals, spec.dims)
    R = 16
    A = gu.rand_factors(spec.dims, R, 3)
    Ad = gu.gpu_factors(A, torch.bfloat16 if bf16 else torch.float32)
    tol = TOL_BF16 if bf16 else TOL_F32
    for mode in (2, 3):
        want = cref.mttkrp(coords, vals, spec.dims, A, mode, nthreads=4)   # fp64 oracle
        t.set_mode_plan(mode, alto.VARIANT_PULL)
        regular = t.mttkrp(mode, Ad, R).cpu().numpy()   # regular entry point; builds the pull lists
        err, bad_zero = ar.row_relative_error(regular, want)
        assert bad_zero == 0 and err <= tol, ("regular", mode, err)
        for call in range(2):
            out = torch.full((spec.dims[mode], R), float("nan"), device="cuda")
            alto.alto_mttkrp_noalloc(t, mode, Ad, R, out)   # element type taken from the factors
            got = out.cpu().numpy()
            err, bad_zero = ar.row_relative_error(got, want)
            assert bad_zero == 0 and err <= tol, ("oracle", mode, call, err)
            err, bad_zero = ar.row_relative_error(got, regular)
            assert bad_zero == 0 and err <= tol, ("regular entry point", mode, call, err)


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
