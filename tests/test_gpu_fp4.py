"""The fused kernel on e2m1 operands (p = 4, S_BR interpolated, CTA pair): the genotypes and the
three e2m1 digits of every fixed-point slice of the per-trait columns, contracted on the
block-scaled FP4 tensor cores.  Each accumulator receives the same integer partial sums as with
bf16 slices, so the outputs must be bitwise equal to the bf16 kernel's (GWAS_FP4=0), and on the
oracle to the mixed path's bar; genotypes outside e2m1's integers keep the bf16 kernel."""
import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem
from tests._metrics import full_b_err, last_coef_err, se_err

pytestmark = pytest.mark.gpu

TOL = 1e-6


def solve(g, P, output, monkeypatch, fp4, i0=0, i1=None, XR=None):
    monkeypatch.setenv("GWAS_FUSED_SHAPE", "2x1x16x1")
    monkeypatch.delenv("GWAS_S_BR", raising=False)
    if fp4:
        monkeypatch.delenv("GWAS_FP4", raising=False)
    else:
        monkeypatch.setenv("GWAS_FP4", "0")
    i1 = P.m if i1 is None else i1
    o = g.gwas_default_opts(precision=g.GWAS_MIXED, output=output)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR if XR is None else XR, P.n)
        M = i1 - i0
        out = np.empty((P.t, M, P.p)) if output == g.GWAS_OUT_FULL_B else np.empty((2, P.t, M), np.float32)
        g.gwas_solve(ctx, P.Y, i0, i1, out)
        info = g.gwas_fp4_info(ctx)
        assert g.gwas_sbr_info(ctx)["terms"] > 0
    finally:
        g.gwas_destroy(ctx)
    return out, info


def same(a, b):
    # bitwise, NaN (singular pairs) included
    return np.array_equal(a.view(np.uint32 if a.dtype == np.float32 else np.uint64),
                          b.view(np.uint32 if b.dtype == np.float32 else np.uint64))


@pytest.mark.parametrize("n,m,t,i0,i1", [(1000, 3000, 100, 0, 3000),   # K one 1024 block set, 5 trait tiles
                                         (300, 1000, 50, 7, 989),      # Kp4 = 512 > Kpad = 320, ragged SNPs
                                         (1100, 700, 30, 0, 700)])     # Kp4 = 1280
def test_fp4_kernel_equals_bf16_kernel_and_oracle(gw, monkeypatch, n, m, t, i0, i1):
    P = make_problem(n, m, t, pm1=3, seed=900 + n)
    got, info = solve(gw, P, gw.GWAS_OUT_LAST_SE, monkeypatch, True, i0, i1)
    ref, info_ref = solve(gw, P, gw.GWAS_OUT_LAST_SE, monkeypatch, False, i0, i1)
    assert info["ready"] and info["launches"] >= 1
    assert not info_ref["ready"] and info_ref["launches"] == 0
    assert same(got, ref)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[i0:i1], P.Y, P.h2)
    beta, s = got[0].T.astype(np.float64), got[1].T.astype(np.float64)
    assert last_coef_err(beta, s, b, se) <= TOL
    assert se_err(s, se) <= TOL


def test_fp4_kernel_full_b(gw, monkeypatch):
    P = make_problem(512, 900, 48, pm1=3, seed=931)
    got, info = solve(gw, P, gw.GWAS_OUT_FULL_B, monkeypatch, True)
    ref, _ = solve(gw, P, gw.GWAS_OUT_FULL_B, monkeypatch, False)
    assert info["launches"] >= 1
    assert same(got, ref)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    assert full_b_err(got.transpose(1, 0, 2), b, se) <= TOL


@pytest.mark.parametrize("value", [5, 7, -5, -8, 9, 127, -128])
def test_genotypes_without_e2m1_codes_keep_the_bf16_kernel(gw, monkeypatch, value):
    # one genotype without an e2m1 code (the integers of e2m1 are 0, +-1, +-2, +-3, +-4 and +-6)
    P = make_problem(256, 600, 40, pm1=3, seed=941)
    XR = P.XR.copy()
    XR[3, 17] = value
    got, info = solve(gw, P, gw.GWAS_OUT_LAST_SE, monkeypatch, True, XR=XR)
    assert not info["ready"] and info["launches"] == 0
    b, se = EigOracle(P.phi, P.XL).solve(XR, P.Y, P.h2)
    beta, s = got[0].T.astype(np.float64), got[1].T.astype(np.float64)
    assert last_coef_err(beta, s, b, se) <= TOL
    # the other e2m1 integers (3, 4, 6 and negatives) have codes: the e2m1 kernel runs, unchanged
    XR2 = P.XR.copy()
    XR2[0, :8] = [3, 4, 6, -1, -2, -6, -3, -4]
    got2, info2 = solve(gw, P, gw.GWAS_OUT_LAST_SE, monkeypatch, True, XR=XR2)
    ref2, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE, monkeypatch, False, XR=XR2)
    assert info2["ready"] and info2["launches"] >= 1
    assert same(got2, ref2)


def solve_budget(g, P, monkeypatch, fp4, budget):
    """solve() with an HBM budget; None when the budget is too small for the call."""
    monkeypatch.setenv("GWAS_FUSED_SHAPE", "2x1x16x1")
    monkeypatch.delenv("GWAS_S_BR", raising=False)
    if fp4:
        monkeypatch.delenv("GWAS_FP4", raising=False)
    else:
        monkeypatch.setenv("GWAS_FP4", "0")
    o = g.gwas_default_opts(precision=g.GWAS_MIXED, output=g.GWAS_OUT_LAST_SE, hbm_budget=int(budget))
    try:
        ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    except g.GwasError as e:
        assert e.code == g.GWAS_ERR_OOM
        return None
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        out = np.empty((2, P.t, P.m), np.float32)
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
        return out, g.gwas_fp4_info(ctx)
    except g.GwasError as e:
        assert e.code == g.GWAS_ERR_OOM
        return None
    finally:
        g.gwas_destroy(ctx)


def test_no_e2m1_copies_under_an_hbm_budget(gw, monkeypatch):
    # the e2m1 genotypes and trait digits are extra device memory that a context's HBM budget did
    # not account for: with a budget the calls run on bf16 operands, with the same results
    P = make_problem(256, 600, 40, pm1=3, seed=951)
    ref, _ = solve_budget(gw, P, monkeypatch, False, 1 << 30)
    got, info = solve_budget(gw, P, monkeypatch, True, 1 << 30)
    assert not info["ready"] and info["launches"] == 0
    assert same(got, ref)
    free, info = solve(gw, P, gw.GWAS_OUT_LAST_SE, monkeypatch, True)
    assert info["ready"] and info["launches"] >= 1
    assert same(free, ref)
