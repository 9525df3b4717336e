"""Parity of the plain FP64 CUDA path with the FP64 oracle (bar: 1e-10)."""
import numpy as np
import pytest

from oracle import EigOracle, direct_gls
from synth import make_problem, genotypes, phenotypes, heritabilities
from tests._metrics import full_b_err, last_coef_err, se_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def run(g, P, output, i0=0, i1=None, trait_block=0, precision=None):
    precision = g.GWAS_FP64 if precision is None else precision
    i1 = P.m if i1 is None else i1
    o = g.gwas_default_opts(precision=precision, output=output, trait_block=trait_block)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        M = i1 - i0
        if output == g.GWAS_OUT_FULL_B:
            out = np.full((P.t, M, P.p), np.nan)
        else:
            out = np.full((2, P.t, M), np.nan, dtype=np.float32)
        rc = g.gwas_solve(ctx, P.Y, i0, i1, out)
        return out, rc, g.gwas_singular_count(ctx)
    finally:
        g.gwas_destroy(ctx)


def oracle(P, i0=0, i1=None):
    i1 = P.m if i1 is None else i1
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[i0:i1], P.Y, P.h2)
    return b, se


@pytest.fixture(scope="module")
def tiny():
    # the smallest workload: n=256, p=4, m=1000, t=10
    return make_problem(256, 1000, 10)


def test_tiny_full_grid_full_b(gw, tiny):
    out, rc, _ = run(gw, tiny, gw.GWAS_OUT_FULL_B)
    assert rc == gw.GWAS_OK
    b, se = oracle(tiny)
    assert full_b_err(out.transpose(1, 0, 2), b, se) <= TOL


def test_tiny_matches_direct_definition(gw, tiny):
    out, rc, _ = run(gw, tiny, gw.GWAS_OUT_FULL_B, 0, 50)
    b, se = direct_gls(tiny.phi, tiny.XL, tiny.XR[:50], tiny.Y, tiny.h2)
    assert full_b_err(out.transpose(1, 0, 2), b, se) <= TOL


def test_tiny_last_se(gw, tiny):
    out, rc, _ = run(gw, tiny, gw.GWAS_OUT_LAST_SE)
    b, se = oracle(tiny)
    beta = out[0].T.astype(np.float64)
    s = out[1].T.astype(np.float64)
    # FP32 output: one rounding of a value computed in FP64
    assert last_coef_err(beta, s, b, se) <= 2 ** -23
    assert se_err(s, se) <= 2 ** -23


@pytest.mark.parametrize("n,m,t,pm1", [(300, 777, 13, 2), (130, 65, 17, 0), (97, 200, 5, 7), (64, 1, 1, 3), (5, 3, 2, 3),
                                       (200, 77, 11, 8), (150, 100, 9, 12), (200, 65, 17, 19), (21, 40, 3, 19)])
def test_ragged_shapes(gw, n, m, t, pm1):
    P = make_problem(n, m, t, pm1=pm1, seed=n + m)
    out, rc, _ = run(gw, P, gw.GWAS_OUT_FULL_B)
    b, se = oracle(P)
    assert full_b_err(out.transpose(1, 0, 2), b, se) <= TOL


def test_snp_range_and_trait_blocks(gw):
    P = make_problem(200, 500, 23, seed=3)
    full, _, _ = run(gw, P, gw.GWAS_OUT_FULL_B)
    part, _, _ = run(gw, P, gw.GWAS_OUT_FULL_B, 123, 391, trait_block=5)
    np.testing.assert_array_equal(part, full[:, 123:391])
    empty, rc, _ = run(gw, P, gw.GWAS_OUT_FULL_B, 7, 7)
    assert rc == gw.GWAS_OK and empty.size == 0


def test_device_pointers(gw):
    import torch
    P = make_problem(256, 300, 12, seed=9)
    ref, _, _ = run(gw, P, gw.GWAS_OUT_FULL_B)
    dev = torch.device("cuda:0")
    o = gw.gwas_default_opts(precision=gw.GWAS_FP64, output=gw.GWAS_OUT_FULL_B)
    ctx = gw.gwas_setup(P.n, P.pm1, torch.from_numpy(P.phi).to(dev), torch.from_numpy(P.XL).to(dev), P.t,
                        torch.from_numpy(P.h2).to(dev), o)
    try:
        gw.gwas_load_snps(ctx, P.m, torch.from_numpy(P.XR).to(dev), P.n)
        out = torch.full((P.t, P.m, P.p), float("nan"), dtype=torch.float64, device=dev)
        gw.gwas_solve(ctx, torch.from_numpy(P.Y).to(dev), 0, P.m, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    finally:
        gw.gwas_destroy(ctx)


def test_singular_pairs_are_flagged(gw):
    P = make_problem(128, 40, 6, seed=4)
    P.XR[17] = 1  # monomorphic SNP: collinear with the intercept column of X_L
    out, rc, cnt = run(gw, P, gw.GWAS_OUT_FULL_B)
    assert rc == gw.GWAS_ERR_SINGULAR_PAIRS and cnt == P.t
    assert np.isnan(out[:, 17]).all()
    b, se = oracle(P, 0, 17)
    assert full_b_err(out[:, :17].transpose(1, 0, 2), b, se) <= TOL


def test_error_codes(gw):
    P = make_problem(64, 10, 3, seed=2)
    o = gw.gwas_default_opts(precision=gw.GWAS_FP64)
    with pytest.raises(gw.GwasError) as e:
        gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, np.array([0.5, 1.5, 0.2]), o)
    assert e.value.code == gw.GWAS_ERR_ARG
    bad = P.phi - 2.0 * np.eye(P.n)  # negative eigenvalues: M_j not SPD at h2 = 1
    with pytest.raises(gw.GwasError) as e:
        gw.gwas_setup(P.n, P.pm1, bad, P.XL, P.t, np.array([1.0, 0.5, 0.2]), o)
    assert e.value.code == gw.GWAS_ERR_NOT_SPD
    XLd = P.XL.copy()
    XLd[2] = XLd[1]  # rank-deficient covariates
    with pytest.raises(gw.GwasError) as e:
        gw.gwas_setup(P.n, P.pm1, P.phi, XLd, P.t, P.h2, o)
    assert e.value.code == gw.GWAS_ERR_ARG
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        with pytest.raises(gw.GwasError) as e:
            gw.gwas_solve(ctx, P.Y, 0, 1, np.zeros((P.t, 1, P.p)))
        assert e.value.code == gw.GWAS_ERR_STATE
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        with pytest.raises(gw.GwasError) as e:
            gw.gwas_solve(ctx, P.Y, 0, P.m + 1, np.zeros((P.t, P.m + 1, P.p)))
        assert e.value.code == gw.GWAS_ERR_ARG
    finally:
        gw.gwas_destroy(ctx)
    small = gw.gwas_default_opts(precision=gw.GWAS_FP64, hbm_budget=4096)
    with pytest.raises(gw.GwasError) as e:
        gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, small)
    assert e.value.code == gw.GWAS_ERR_OOM


def test_sampled_pairs_at_fp64_vs_fp32_workload_size(gw):
    # n=1000, p=4, m=100,000, t=1,000 (full b in FP64); the oracle checks a sample of SNPs
    n, m, t = 1000, 100_000, 1000
    P = make_problem(n, m, t)
    o = gw.gwas_default_opts(precision=gw.GWAS_FP64, output=gw.GWAS_OUT_FULL_B)
    ctx = gw.gwas_setup(n, 3, P.phi, P.XL, t, P.h2, o)
    try:
        gw.gwas_load_snps(ctx, m, P.XR, n)
        out = np.empty((t, m, 4))
        assert gw.gwas_solve(ctx, P.Y, 0, m, out) == gw.GWAS_OK
    finally:
        gw.gwas_destroy(ctx)
    rng = np.random.default_rng(0)
    idx = np.concatenate([np.arange(32), m - 32 + np.arange(32), rng.choice(m, 64, replace=False)])
    tj = np.concatenate([np.arange(8), rng.choice(t, 24, replace=False)])
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[idx], P.Y[tj], P.h2[tj])
    got = out[tj][:, idx].transpose(1, 0, 2)
    assert full_b_err(got, b, se) <= TOL
