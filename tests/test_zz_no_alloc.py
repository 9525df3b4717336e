"""The allocation-free entry point gives the same results as gwas_solve.

gwas_solve_fp64_noalloc serves callers that cannot allocate device memory (their
host application's memory manager owns the device, or they are plug-in code handed
only buffers and a stream).  It must agree with the regular FP64 path, call after
call, although every call reuses the same fixed scratch array.  This file is
collected last so that a run stopping at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

from synth import make_problem
from tests._metrics import full_b_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def regular(g, P, output):
    o = g.gwas_default_opts(precision=g.GWAS_FP64, output=output)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        out = np.empty((P.t, P.m, P.p)) if output == g.GWAS_OUT_FULL_B else np.empty((2, P.t, P.m), np.float32)
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
        return out
    finally:
        g.gwas_destroy(ctx)


def rotated_inputs(P, dev):
    import torch
    lam, Z = np.linalg.eigh(P.phi)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return (to(lam), to(P.XL @ Z), to(P.XR.astype(np.float64) @ Z), to(P.Y @ Z), to(P.h2))


def test_noalloc_matches_gwas_solve_twice(gw):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    problems = [make_problem(256, 500, 24, seed=31), make_problem(200, 333, 17, seed=32),
                make_problem(120, 70, 9, pm1=19, seed=34)]  # p = 20, the top of the paper's range
    for P in problems:  # two calls in a row, the second on other data and sizes
        ref = regular(gw, P, gw.GWAS_OUT_FULL_B)
        lam, XLt, Xt, Yt, h2 = rotated_inputs(P, dev)
        out = torch.full((P.t, P.m, P.p), float("nan"), dtype=torch.float64, device=dev)
        rc, sing = gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lam, XLt, Xt, P.m, Yt, h2, P.t, gw.GWAS_OUT_FULL_B, out)
        assert rc == gw.GWAS_OK and sing == 0
        got = out.cpu().numpy()
        se = regular(gw, P, gw.GWAS_OUT_LAST_SE)[1].T.astype(np.float64)
        assert full_b_err(got.transpose(1, 0, 2), ref.transpose(1, 0, 2), se) <= TOL


def test_noalloc_last_se_and_singular_pairs(gw):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    P = make_problem(128, 90, 9, seed=33)
    P.XR[5] = 1  # monomorphic SNP: its pairs are singular
    ref = regular(gw, P, gw.GWAS_OUT_LAST_SE)
    lam, XLt, Xt, Yt, h2 = rotated_inputs(P, dev)
    for _ in range(2):
        out = torch.full((2, P.t, P.m), float("nan"), dtype=torch.float32, device=dev)
        rc, sing = gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lam, XLt, Xt, P.m, Yt, h2, P.t, gw.GWAS_OUT_LAST_SE, out)
        assert rc == gw.GWAS_ERR_SINGULAR_PAIRS and sing == P.t
        got = out.cpu().numpy()
        assert np.isnan(got[:, :, 5]).all()
        keep = np.r_[0:5, 6:P.m]
        beta, se = got[0][:, keep].astype(np.float64), got[1][:, keep].astype(np.float64)
        rb, rs = ref[0][:, keep].astype(np.float64), ref[1][:, keep].astype(np.float64)
        assert np.max(np.abs(beta - rb) / np.maximum(np.abs(rb), rs)) <= 2 ** -22
        assert np.max(np.abs(se - rs) / rs) <= 2 ** -22


def test_noalloc_rejects_sizes_beyond_its_scratch(gw):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    n, pm1, t, m = 2000, 3, 200, 4  # 200 * 5 * 2000 doubles = 16 MB > 8 MiB
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device=dev)
    with pytest.raises(gw.GwasError) as e:
        gw.gwas_solve_fp64_noalloc(n, pm1, z(n), z(pm1, n), z(m, n), m, z(t, n), z(t), t, gw.GWAS_OUT_FULL_B,
                                   z(t, m, pm1 + 1))
    assert e.value.code == gw.GWAS_ERR_UNSUPPORTED
