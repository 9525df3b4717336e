"""The eigendecomposition of gwas_setup: the FP32 eigensolver refined to FP64 accuracy (the
iteration of Ogita and Aishima, with FP64-accurate products on the tensor cores) against the FP64
eigensolver (GWAS_EIG=fp64) and the oracle, through the FP64 path's full b (bar 1e-10).

Cases: kinships of several sizes, from n = 5 to a large one with a degenerate eigenvalue cluster
(fewer kinship markers than individuals: 1100 eigenvalues equal to the ridge), and heritabilities
that include 0 and 1, where M_j = Phi and its conditioning (up to ~10^4 here) amplifies any error
in Z or Lambda."""
import dataclasses

import numpy as np
import pytest

from oracle import EigOracle
from synth import kinship, make_problem
from tests._metrics import full_b_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def run(g, P, monkeypatch, fp64_eig):
    if fp64_eig:
        monkeypatch.setenv("GWAS_EIG", "fp64")
    else:
        monkeypatch.delenv("GWAS_EIG", raising=False)
    o = g.gwas_default_opts(precision=g.GWAS_FP64, output=g.GWAS_OUT_FULL_B)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        steps = g.gwas_eig_info(ctx)
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        out = np.full((P.t, P.m, P.p), np.nan)
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
    finally:
        g.gwas_destroy(ctx)
    return out, steps


@pytest.mark.parametrize("n,snps,pm1", [(5, 5000, 1), (21, 5000, 3), (300, 5000, 3), (1000, 5000, 3),
                                        (1500, 400, 3)])
def test_refined_eigendecomposition_matches_fp64_solver_and_oracle(gw, monkeypatch, n, snps, pm1):
    P = make_problem(n, 150, 10, pm1=pm1, seed=700 + n)
    h2 = P.h2.copy()
    h2[:4] = [0.0, 0.5, 0.999, 1.0]
    XR = P.XR.copy()
    mono = np.flatnonzero(XR.min(axis=1) == XR.max(axis=1))
    XR[mono, 0] = (XR[mono, 0] + 1) % 3   # a monomorphic SNP makes X_i singular at small n
    P = dataclasses.replace(P, phi=kinship(n, seed=700 + n, snps=snps), h2=h2, XR=XR)
    got, steps = run(gw, P, monkeypatch, fp64_eig=False)
    ref, steps_ref = run(gw, P, monkeypatch, fp64_eig=True)
    assert 0 <= steps <= 8, "the refinement fell back to the FP64 solver"
    assert steps_ref == -1
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    assert full_b_err(np.transpose(got, (1, 0, 2)), b, se) <= TOL
    assert full_b_err(np.transpose(ref, (1, 0, 2)), b, se) <= TOL
    assert full_b_err(np.transpose(got, (1, 0, 2)), np.transpose(ref, (1, 0, 2)), se) <= TOL


def test_refined_eigendecomposition_in_the_mixed_path(gw, monkeypatch):
    # the mixed path on the same kinship gives the same results from either decomposition
    P = make_problem(1000, 2000, 40, seed=731)
    outs = []
    for fp64_eig in (False, True):
        if fp64_eig:
            monkeypatch.setenv("GWAS_EIG", "fp64")
        else:
            monkeypatch.delenv("GWAS_EIG", raising=False)
        o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
        ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
        try:
            assert (gw.gwas_eig_info(ctx) >= 0) != fp64_eig
            gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
            out = np.empty((2, P.t, P.m), np.float32)
            gw.gwas_solve(ctx, P.Y, 0, P.m, out)
        finally:
            gw.gwas_destroy(ctx)
        outs.append(out.astype(np.float64))
    a, r = outs
    assert np.max(np.abs(a[0] - r[0]) / np.maximum(np.abs(r[0]), r[1])) <= 1e-6
    assert np.max(np.abs(a[1] - r[1]) / r[1]) <= 1e-6


def test_larger_kinships_go_to_the_fp64_solver(gw):
    # above n = 2048 the refinement's steps were measured not to converge: the FP64 solver runs
    # directly
    n = 2049
    phi, XL = kinship(n, seed=777), make_problem(n, 1, 1, seed=777, with_snps=False).XL
    o = gw.gwas_default_opts(precision=gw.GWAS_FP64)
    ctx = gw.gwas_setup(n, 3, phi, XL, 1, np.array([0.5]), o)
    try:
        assert gw.gwas_eig_info(ctx) == -1
    finally:
        gw.gwas_destroy(ctx)
