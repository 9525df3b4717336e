"""S_BR from its Chebyshev series in h^2 (the mixed path's default where the bound allows it)
against the same solve with S_BR contracted per pair (GWAS_S_BR=exact) and against the oracle:
both output modes, several p (one-CTA tiles of 32, 16 and 8 traits), ragged SNP ranges, a
change of heritabilities (the plan is redone), and the fall-back when no plan meets the bound."""
import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem
from tests._metrics import full_b_err, last_coef_err, se_err

pytestmark = pytest.mark.gpu

TOL = 1e-6


def solve(g, P, output, i0=0, i1=None, h2=None, exact=False, monkeypatch=None):
    i1 = P.m if i1 is None else i1
    if monkeypatch is not None:
        if exact:
            monkeypatch.setenv("GWAS_S_BR", "exact")
        else:
            monkeypatch.delenv("GWAS_S_BR", raising=False)
    o = g.gwas_default_opts(precision=g.GWAS_MIXED, output=output)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2 if h2 is None else h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        M = i1 - i0
        out = np.empty((P.t, M, P.p)) if output == g.GWAS_OUT_FULL_B else np.empty((2, P.t, M), np.float32)
        g.gwas_solve(ctx, P.Y, i0, i1, out)
        info = g.gwas_sbr_info(ctx)
    finally:
        g.gwas_destroy(ctx)
    return out, info


@pytest.mark.parametrize("pm1", [3, 1, 7, 11, 19])
def test_interpolated_sbr_matches_exact_and_oracle(gw, monkeypatch, pm1):
    P = make_problem(300, 700, 70 if pm1 < 8 else 37, pm1=pm1, seed=500 + pm1)
    i0, i1 = 5, 689  # ragged at both ends
    got, info = solve(gw, P, gw.GWAS_OUT_LAST_SE, i0, i1, monkeypatch=monkeypatch)
    ex, info_ex = solve(gw, P, gw.GWAS_OUT_LAST_SE, i0, i1, exact=True, monkeypatch=monkeypatch)
    assert 4 <= info["terms"] <= 24 and info["bound"] <= 1e-10
    assert info["lo"] <= P.h2.min() and info["hi"] >= P.h2.max()
    assert info_ex["terms"] == 0
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[i0:i1], P.Y, P.h2)
    for out in (got, ex):
        beta, s = out[0].T.astype(np.float64), out[1].T.astype(np.float64)
        assert last_coef_err(beta, s, b, se) <= TOL
        assert se_err(s, se) <= TOL
    # the two ways of obtaining S_BR agree to the same bar
    bg, be = got[0].T.astype(np.float64), ex[0].T.astype(np.float64)
    assert np.max(np.abs(bg - be) / np.maximum(np.abs(be), ex[1].T)) <= TOL


@pytest.mark.parametrize("pm1", [3, 10])
def test_interpolated_sbr_full_b(gw, monkeypatch, pm1):
    P = make_problem(256, 400, 40, pm1=pm1, seed=520 + pm1)
    got, info = solve(gw, P, gw.GWAS_OUT_FULL_B, monkeypatch=monkeypatch)
    assert info["terms"] > 0
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    assert full_b_err(got.transpose(1, 0, 2), b, se) <= TOL


def test_plan_follows_the_heritabilities(gw, monkeypatch):
    """A narrow range of heritabilities needs fewer terms than a wide one; after gwas_set_h2 the
    plan is redone for the new range and the results stay on the oracle."""
    monkeypatch.delenv("GWAS_S_BR", raising=False)
    P = make_problem(200, 300, 24, seed=530)
    narrow = np.linspace(0.40, 0.42, P.t)
    wide = np.linspace(0.0, 1.0, P.t)
    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, narrow, o)
    oracle = EigOracle(P.phi, P.XL)
    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        infos = []
        for h2 in (narrow, wide):
            gw.gwas_set_h2(ctx, P.t, h2)
            out = np.empty((2, P.t, P.m), np.float32)
            gw.gwas_solve(ctx, P.Y, 0, P.m, out)
            info = gw.gwas_sbr_info(ctx)
            infos.append(info)
            assert info["lo"] <= h2.min() + 1e-12 and info["hi"] >= h2.max() - 1e-12
            b, se = oracle.solve(P.XR, P.Y, h2)
            beta, s = out[0].T.astype(np.float64), out[1].T.astype(np.float64)
            assert last_coef_err(beta, s, b, se) <= TOL and se_err(s, se) <= TOL
    finally:
        gw.gwas_destroy(ctx)
    assert 0 < infos[0]["terms"] < infos[1]["terms"]


def test_no_covariates_falls_back_to_the_contraction(gw, monkeypatch):
    """p = 1: the SNPs are not centred, so they reach the kinship's 1e-3 eigenvalue, whose pole
    sits just above h^2 = 1; with heritabilities up to 0.999 no plan of <= 24 terms meets the
    bound and S_BR is contracted per pair."""
    monkeypatch.delenv("GWAS_S_BR", raising=False)
    P = make_problem(160, 250, 20, pm1=0, seed=540)
    h2 = np.linspace(0.0, 0.999, P.t)
    got, info = solve(gw, P, gw.GWAS_OUT_LAST_SE, h2=h2)
    assert info["terms"] == 0
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, h2)
    beta, s = got[0].T.astype(np.float64), got[1].T.astype(np.float64)
    assert last_coef_err(beta, s, b, se) <= TOL and se_err(s, se) <= TOL


def test_interpolated_sbr_in_the_cta_pair_shape(gw, monkeypatch):
    """The CTA-pair launch shape (p = 4) with S_BR interpolated: each CTA of the pair streams its
    own SNP rows and half of the C1 trait rows; an odd number of SNP tiles leaves the second CTA
    of the last pair without a tile."""
    monkeypatch.delenv("GWAS_S_BR", raising=False)
    monkeypatch.setenv("GWAS_FUSED_SHAPE", "2x1x16x1")
    P = make_problem(333, 5 * 128 + 77, 75, seed=550)
    got, info = solve(gw, P, gw.GWAS_OUT_LAST_SE, 3, P.m - 2)
    assert info["terms"] > 0
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[3:P.m - 2], P.Y, P.h2)
    beta, s = got[0].T.astype(np.float64), got[1].T.astype(np.float64)
    assert last_coef_err(beta, s, b, se) <= TOL and se_err(s, se) <= TOL
    full, _ = solve(gw, P, gw.GWAS_OUT_FULL_B)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    assert full_b_err(full.transpose(1, 0, 2), b, se) <= TOL
