"""Parity of the mixed-precision tensor-core path with the FP64 oracle.

Bar: relative error <= 1e-6 on the SNP coefficient, measured against
max(|b*|, SE*) (the coefficients of pure-noise traits scatter around zero), and
<= 1e-6 relative on its standard error.
"""
import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem, genotypes, phenotypes, heritabilities, kinship, covariates
from tests._metrics import full_b_err, last_coef_err, se_err

pytestmark = pytest.mark.gpu

TOL = 1e-6


def solve(g, P, output, i0=0, i1=None, trait_block=0, precision=None):
    precision = g.GWAS_MIXED if precision is None else precision
    i1 = P.m if i1 is None else i1
    o = g.gwas_default_opts(precision=precision, output=output, trait_block=trait_block)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        M = i1 - i0
        out = np.full((P.t, M, P.p), np.nan) if output == g.GWAS_OUT_FULL_B else \
            np.full((2, P.t, M), np.nan, dtype=np.float32)
        rc = g.gwas_solve(ctx, P.Y, i0, i1, out)
        return out, rc, g.gwas_singular_count(ctx)
    finally:
        g.gwas_destroy(ctx)


def check_last(out, b, se, tol=TOL):
    beta = out[0].T.astype(np.float64)
    s = out[1].T.astype(np.float64)
    e1, e2 = last_coef_err(beta, s, b, se), se_err(s, se)
    assert e1 <= tol and e2 <= tol, (e1, e2)
    return e1, e2


@pytest.mark.parametrize("n,m,t", [(256, 1000, 10), (300, 777, 45), (1000, 300, 70), (130, 129, 33)])
def test_last_se_parity(gw, n, m, t):
    P = make_problem(n, m, t, seed=n * 7 + m)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_OK
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check_last(out, b, se)


def test_full_b_parity(gw):
    P = make_problem(256, 400, 40, seed=21)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    err = full_b_err(out.transpose(1, 0, 2), b, se)
    assert err <= TOL, err


def test_range_and_blocks_are_bitwise_stable(gw):
    P = make_problem(200, 700, 70, seed=5)
    full, _, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    part, _, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE, 133, 601, trait_block=33)
    np.testing.assert_array_equal(part, full[:, :, 133:601])


def test_singular_snp(gw):
    P = make_problem(128, 60, 6, seed=4)
    P.XR[17] = 2
    out, rc, cnt = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_ERR_SINGULAR_PAIRS and cnt == P.t
    assert np.isnan(out[:, :, 17]).all()
    keep = np.r_[0:17, 18:P.m]
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[keep], P.Y, P.h2)
    check_last(out[:, :, keep], b, se)


def test_mixed_matches_fp64_gpu(gw):
    P = make_problem(512, 2000, 64, seed=8)
    mixed, _, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    fp64, _, _ = solve(gw, P, gw.GWAS_OUT_FULL_B, precision=gw.GWAS_FP64)
    b = fp64.transpose(1, 0, 2)
    _, se_ref = EigOracle(P.phi, P.XL).solve(P.XR[:1], P.Y, P.h2)
    # SE of the FP64 path from its own LAST_SE run
    fse, _, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE, precision=gw.GWAS_FP64)
    check_last(mixed, b, fse[1].T.astype(np.float64))


def test_mixed_matches_fp64_gpu_on_workload_slice(gw):
    """Every pair of SNPs [0, 16384) x all 10,000 traits of the n=1000, p=4 workload: the mixed
    path against the FP64 GPU path (itself pinned to the oracle at 1e-10), compared on the device."""
    torch = pytest.importorskip("torch")
    n, M, t = 1000, 16384, 10_000
    dev = torch.device("cuda:0")
    phi, XL, h2 = kinship(n), covariates(n), heritabilities(t)
    XR = torch.from_numpy(genotypes(n, 1_000_000, i0=0, i1=M)).to(dev)
    Y = torch.from_numpy(phenotypes(n, t)).to(dev)
    outs = {}
    for prec in (gw.GWAS_MIXED, gw.GWAS_FP64):
        o = gw.gwas_default_opts(precision=prec, output=gw.GWAS_OUT_LAST_SE)
        ctx = gw.gwas_setup(n, 3, phi, XL, t, h2, o)
        try:
            gw.gwas_load_snps(ctx, M, XR, n)
            out = torch.full((2, t, M), float("nan"), dtype=torch.float32, device=dev)
            assert gw.gwas_solve(ctx, Y, 0, M, out) == gw.GWAS_OK
            outs[prec] = out.double()
        finally:
            gw.gwas_destroy(ctx)
    (bm, sm), (b64, s64) = outs[gw.GWAS_MIXED], outs[gw.GWAS_FP64]
    assert bool(torch.isfinite(bm).all()) and bool(torch.isfinite(sm).all())
    err_b = ((bm - b64).abs() / torch.maximum(b64.abs(), s64)).max().item()
    err_se = ((sm - s64).abs() / s64).max().item()
    assert err_b <= TOL and err_se <= TOL, (err_b, err_se)


def test_sampled_pairs_at_full_mixed_workload(gw):
    """n=1000, p=4, m=1,000,000, t=10,000 on the device; the oracle checks sampled pairs."""
    torch = pytest.importorskip("torch")
    n, m, t = 1000, 1_000_000, 10_000
    dev = torch.device("cuda:0")
    phi, XL, h2 = kinship(n), covariates(n), heritabilities(t)
    XR = genotypes(n, m)
    Y = phenotypes(n, t)
    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
    ctx = gw.gwas_setup(n, 3, phi, XL, t, h2, o)
    try:
        gw.gwas_load_snps(ctx, m, torch.from_numpy(XR).to(dev), n)
        out = torch.empty((2, t, m), dtype=torch.float32, device=dev)
        assert gw.gwas_solve(ctx, torch.from_numpy(Y).to(dev), 0, m, out) == gw.GWAS_OK
        rng = np.random.default_rng(1)
        idx = np.unique(np.concatenate([np.arange(64), m - 64 + np.arange(64), rng.choice(m, 256, replace=False)]))
        tj = np.unique(np.concatenate([np.arange(16), t - 16 + np.arange(16), rng.choice(t, 64, replace=False)]))
        it, jt = torch.from_numpy(idx).to(dev), torch.from_numpy(tj).to(dev)
        got = out[:, jt][:, :, it].cpu().numpy()
        finite = bool(torch.isfinite(out).all().item())
    finally:
        gw.gwas_destroy(ctx)
    assert finite
    b, se = EigOracle(phi, XL).solve(XR[idx], Y[tj], h2[tj])
    check_last(got, b, se)


# p - 1 up to 19 (Section 3: 2 <= p <= 20): trait tiles of 32 (p - 1 <= 3), 16 (<= 10) and 8;
# the trait and SNP counts leave ragged last tiles.
@pytest.mark.parametrize("pm1,n,m,t", [(0, 200, 300, 40), (1, 256, 257, 33), (2, 300, 200, 17), (4, 256, 300, 20),
                                       (5, 130, 129, 45), (6, 200, 256, 19), (7, 97, 300, 35), (8, 200, 300, 37),
                                       (10, 160, 257, 33), (11, 200, 300, 21), (13, 130, 129, 17), (16, 256, 200, 9),
                                       (19, 200, 300, 25)])
def test_general_p_last_se(gw, pm1, n, m, t):
    P = make_problem(n, m, t, pm1=pm1, seed=101 * pm1 + n)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_OK
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check_last(out, b, se)


@pytest.mark.parametrize("pm1", [0, 2, 5, 7, 10, 11, 19])
def test_general_p_full_b(gw, pm1):
    P = make_problem(160, 290, 37, pm1=pm1, seed=7 + pm1)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B)
    assert rc == gw.GWAS_OK
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    err = full_b_err(out.transpose(1, 0, 2), b, se)
    assert err <= TOL, err


# One trait: the single-trait (GEMV-shaped, HBM-bound) kernel instead of the fused one.
@pytest.mark.parametrize("pm1", [0, 3, 7, 12, 19])
def test_single_trait(gw, pm1):
    P = make_problem(300, 1500, 1, pm1=pm1, seed=83 + pm1)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_OK
    check_last(out, b, se)
    full, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B)
    assert full_b_err(full.transpose(1, 0, 2), b, se) <= TOL
    # an unaligned SNP range
    part, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE, 77, 1333)
    check_last(part, b[77:1333], se[77:1333])


def test_single_trait_blocks_match_the_oracle(gw):
    # trait blocks of one trait: every block runs the single-trait kernel
    P = make_problem(256, 900, 9, seed=84)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE, trait_block=1)
    assert rc == gw.GWAS_OK
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check_last(out, b, se)


def test_single_trait_singular_snp(gw):
    P = make_problem(128, 300, 1, seed=85)
    P.XR[40] = 1
    out, rc, cnt = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_ERR_SINGULAR_PAIRS and cnt == 1
    assert np.isnan(out[0, 0, 40]) and np.isnan(out[1, 0, 40])
    ok = np.ones(P.m, bool)
    ok[40] = False
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[ok], P.Y, P.h2)
    check_last(out[:, :, ok], b, se)


def test_largest_n_of_the_paper(gw):
    # n = 10^4, the top of the paper's range (Section 3): the slice scales and the exactness
    # bound of the level-0 sums (512 n < 2^24 for C1) at their largest; FP64 path alongside
    P = make_problem(10_000, 260, 12, seed=2024)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_OK
    check_last(out, b, se)
    full, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B)
    assert full_b_err(full.transpose(1, 0, 2), b, se) <= TOL
    full64, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B, precision=gw.GWAS_FP64)
    assert full_b_err(full64.transpose(1, 0, 2), b, se) <= 1e-10


def test_host_output_in_growing_blocks(gw):
    # a host output is solved in trait blocks growing from tb/8 (here 32, 64, 64, 40 traits);
    # every pair's result is the same as with one device-side block
    import torch
    P = make_problem(256, 700, 200, seed=2025)
    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE, trait_block=64)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        dev = torch.full((2, P.t, P.m), float("nan"), dtype=torch.float32, device="cuda:0")
        gw.gwas_solve(ctx, P.Y, 0, P.m, dev)
        pinned = torch.full((2, P.t, P.m), float("nan"), dtype=torch.float32).pin_memory()
        gw.gwas_solve(ctx, P.Y, 0, P.m, pinned)
        pageable = np.full((2, P.t, P.m), np.nan, dtype=np.float32)
        gw.gwas_solve(ctx, P.Y, 0, P.m, pageable)
    finally:
        gw.gwas_destroy(ctx)
    ref = dev.cpu().numpy()
    np.testing.assert_array_equal(pinned.numpy(), ref)
    np.testing.assert_array_equal(pageable, ref)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check_last(ref, b, se)


@pytest.mark.parametrize("precision,output", [("mixed", "last"), ("mixed", "full"), ("fp64", "last")])
def test_page_locked_output_direct_and_staged(gw, monkeypatch, precision, output):
    # a page-locked host output is stored by the kernels themselves where the device reads the
    # CPU's page tables, else (and with GWAS_HOST_OUTPUT=staged) copied through device staging;
    # both give the device output bit for bit
    import torch
    P = make_problem(200, 650, 70, pm1=4, seed=2027)
    prec = gw.GWAS_MIXED if precision == "mixed" else gw.GWAS_FP64
    out_kind = gw.GWAS_OUT_LAST_SE if output == "last" else gw.GWAS_OUT_FULL_B
    shape, dt = ((2, P.t, P.m), torch.float32) if output == "last" else ((P.t, P.m, P.p), torch.float64)
    o = gw.gwas_default_opts(precision=prec, output=out_kind, trait_block=32)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        dev = torch.full(shape, float("nan"), dtype=dt, device="cuda:0")
        gw.gwas_solve(ctx, P.Y, 0, P.m, dev)
        direct = torch.full(shape, float("nan"), dtype=dt).pin_memory()
        gw.gwas_solve(ctx, P.Y, 0, P.m, direct)
        monkeypatch.setenv("GWAS_HOST_OUTPUT", "staged")
        staged = torch.full(shape, float("nan"), dtype=dt).pin_memory()
        gw.gwas_solve(ctx, P.Y, 0, P.m, staged)
        monkeypatch.delenv("GWAS_HOST_OUTPUT")
        # a sub-range of SNPs into a page-locked array sized for it
        part = torch.full((2, P.t, 300) if output == "last" else (P.t, 300, P.p), float("nan"), dtype=dt).pin_memory()
        gw.gwas_solve(ctx, P.Y, 100, 400, part)
    finally:
        gw.gwas_destroy(ctx)
    ref = dev.cpu().numpy()
    np.testing.assert_array_equal(direct.numpy(), ref)
    np.testing.assert_array_equal(staged.numpy(), ref)
    np.testing.assert_array_equal(part.numpy(), ref[:, :, 100:400] if output == "last" else ref[:, 100:400])
    assert np.isfinite(ref).all()


@pytest.mark.parametrize("offset", [0, 1])
def test_page_locked_genotypes_read_directly(gw, monkeypatch, offset):
    # page-locked host genotypes are read by the conversion kernel itself where the device reads
    # the CPU's page tables, else (and with GWAS_HOST_INPUT=staged) copied first; both give the
    # results of device genotypes bit for bit, also from a buffer that starts off an 8-byte boundary
    import torch
    P = make_problem(301, 1500, 40, seed=2031)
    flat = torch.zeros(P.m * P.n + 8, dtype=torch.int8).pin_memory()
    pinned = flat[offset:offset + P.m * P.n].view(P.m, P.n)
    pinned.copy_(torch.from_numpy(P.XR))
    outs = []
    for XR, mode in ((torch.from_numpy(P.XR).cuda(), None), (pinned, None), (pinned, "staged")):
        if mode:
            monkeypatch.setenv("GWAS_HOST_INPUT", mode)
        else:
            monkeypatch.delenv("GWAS_HOST_INPUT", raising=False)
        o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
        ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
        try:
            gw.gwas_load_snps(ctx, P.m, XR, P.n)
            out = np.full((2, P.t, P.m), np.nan, dtype=np.float32)
            gw.gwas_solve(ctx, P.Y, 0, P.m, out)
        finally:
            gw.gwas_destroy(ctx)
        outs.append(out)
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])
    b, se = EigOracle(P.phi, P.XL).solve(P.XR[:200], P.Y, P.h2)
    check_last(outs[0][:, :, :200], b, se)


def test_extreme_heritabilities(gw):
    # h^2 over the whole range of the model, both ends included: M_j = I (ordinary least
    # squares) at 0 and M_j = Phi at 1; near 1 the weights e_j = 1/(h^2 lambda + 1 - h^2)
    # spread over three orders of magnitude
    P = make_problem(300, 400, 8, seed=2026)
    P.h2[:] = [0.0, 1e-3, 0.5, 0.9, 0.95, 0.99, 0.999, 1.0]
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_OK
    beta, s = out[0].T.astype(np.float64), out[1].T.astype(np.float64)
    errs = [last_coef_err(beta[:, j:j + 1], s[:, j:j + 1], b[:, j:j + 1], se[:, j:j + 1]) for j in range(P.t)]
    serrs = [se_err(s[:, j:j + 1], se[:, j:j + 1]) for j in range(P.t)]
    assert max(errs) <= TOL and max(serrs) <= TOL, (errs, serrs)
    full64, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B, precision=gw.GWAS_FP64)
    assert full_b_err(full64.transpose(1, 0, 2), b, se) <= 1e-10


@pytest.mark.parametrize("n,m,t,pm1", [(8, 1, 1, 3), (30, 1, 40, 3), (64, 129, 1, 0), (64, 300, 33, 19), (1000, 1, 1, 3),
                                       (70, 5, 2, 1)])
def test_degenerate_shapes(gw, n, m, t, pm1):
    # one SNP, one trait, few degrees of freedom (4 at n = 8, 44 at p = 20), n below one K block
    # of 64 and not a multiple of it; both output modes against the oracle.  (With n - p of 1 or
    # 2, RSS = rr - num beta can be a tiny difference for some pairs and the FP32 epilogue's SE
    # loses its relative accuracy there; the FP64 path covers that regime, far below the paper's
    # n >= 10^3.)
    P = make_problem(n, m, t, pm1=pm1, seed=5000 + n + m + t)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    assert rc == gw.GWAS_OK
    check_last(out, b, se)
    full, rc, _ = solve(gw, P, gw.GWAS_OUT_FULL_B)
    assert full_b_err(full.transpose(1, 0, 2), b, se) <= TOL
    empty, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE, 0, 0)
    assert rc == gw.GWAS_OK and empty.size == 0


def _conditioning(P):
    """kappa[i, j] = rr_j / RSS_ij in FP64: the whitened residual of y_j on X_L over that on
    [X_L | x_i].  The SE is sqrt(RSS / ((n - p) delta)) with RSS = rr - num^2 / delta, so a relative
    error eps in num^2 / delta moves the SE by about eps * kappa / 2."""
    lam, Z = np.linalg.eigh(P.phi)
    kap = np.empty((P.m, P.t))
    for j in range(P.t):
        e = 1.0 / (P.h2[j] * lam + 1.0 - P.h2[j])
        W = (Z * e) @ Z.T                                  # M_j^-1
        XL = P.XL.T
        y = P.Y[j]

        def rss(X):
            A = X.T @ W @ X
            bb = np.linalg.solve(A, X.T @ W @ y)
            r = y - X @ bb
            return r @ W @ r

        rr = rss(XL)
        for i in range(P.m):
            kap[i, j] = rr / rss(np.column_stack([XL, P.XR[i].astype(np.float64)]))
    return kap


@pytest.mark.parametrize("n,pm1", [(5, 3), (21, 19), (6, 3), (22, 19)])
def test_one_and_two_degrees_of_freedom(gw, n, pm1):
    """n - p of 1 and 2 on the mixed path: the SNP coefficient stays within the 1e-6 bar; the SE
    stays within 1e-6 where rr / RSS <= 2 (the residual is not a small difference), and elsewhere within a bound
    proportional to rr / RSS (the conditioning of RSS = rr - num^2 / delta: about 1e-7 relative
    error in num^2 / delta from the slices, whatever precision the subtraction is done in)."""
    P = make_problem(n, 150, 30, pm1=pm1, seed=7000 + n + pm1)
    # a handful of individuals leaves many SNPs monomorphic (no solution, NaN by design); make
    # every SNP polymorphic so that every pair has a unique solution to compare
    mono = P.XR.min(axis=1) == P.XR.max(axis=1)
    P.XR[mono, 0] = (P.XR[mono, 0] + 1) % 3
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    out, rc, _ = solve(gw, P, gw.GWAS_OUT_LAST_SE)
    bl = b[..., -1]
    beta, s = out[0].T.astype(np.float64), out[1].T.astype(np.float64)
    ok = np.isfinite(bl) & np.isfinite(se) & (se > 0)
    assert ok.mean() > 0.9
    assert np.all(np.isfinite(beta[ok])) and np.all(s[ok] > 0)
    assert np.max(np.abs(beta - bl)[ok] / np.maximum(np.abs(bl), se)[ok]) <= TOL
    kap = _conditioning(P)
    rel = np.abs(s - se) / se
    assert np.all(rel[ok] <= TOL + 1e-6 * kap[ok])
    well = ok & (kap <= 2)
    assert well.sum() > 0 and np.max(rel[well]) <= TOL
