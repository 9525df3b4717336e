"""Failure detection without a GPU fault: a kernel wait that nothing completes gives up
after its limit and reports it, and the device stays usable afterwards."""
import numpy as np
import pytest

from synth import make_problem

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(gw):
    for limit in (0.02, 0.2):
        rc, waited = gw.gwas_check_bounded_wait(0, limit)
        assert rc == gw.GWAS_ERR_TIMEOUT
        assert 0 < waited < limit + 0.5
    P = make_problem(128, 64, 4, seed=1)
    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        out = np.empty((2, P.t, P.m), np.float32)
        assert gw.gwas_solve(ctx, P.Y, 0, P.m, out) == gw.GWAS_OK
        assert np.isfinite(out).all()
    finally:
        gw.gwas_destroy(ctx)


def test_bounded_wait_rejects_bad_limits(gw):
    assert gw.gwas_check_bounded_wait(0, 0.0)[0] == gw.GWAS_ERR_ARG
    assert gw.gwas_check_bounded_wait(0, 60.0)[0] == gw.GWAS_ERR_ARG
