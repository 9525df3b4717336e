"""The allocation-free entry point gives the same results as gwas_solve and the oracle.

gwas_solve_fp64_noalloc serves callers that cannot allocate device memory (their
host application's memory manager owns the device, or they are plug-in code handed
only buffers and a stream).  It must agree with the regular FP64 path, call after
call, although every call reuses the same fixed scratch array.  This file is
collected last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem
from tests._metrics import full_b_err, last_coef_err, se_err

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
        # and directly against the CPU oracle (FP64, the plain definition in GEMM form)
        b_o, se_o = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
        assert full_b_err(got.transpose(1, 0, 2), b_o, se_o) <= TOL


def test_noalloc_last_se_against_the_oracle(gw):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    P = make_problem(300, 260, 21, seed=35)
    lam, XLt, Xt, Yt, h2 = rotated_inputs(P, dev)
    out = torch.full((2, P.t, P.m), float("nan"), dtype=torch.float32, device=dev)
    rc, sing = gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lam, XLt, Xt, P.m, Yt, h2, P.t, gw.GWAS_OUT_LAST_SE, out)
    assert rc == gw.GWAS_OK and sing == 0
    got = out.cpu().numpy()
    b_o, se_o = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    beta, se = got[0].T.astype(np.float64), got[1].T.astype(np.float64)
    assert last_coef_err(beta, se, b_o, se_o) <= 2 ** -22 and se_err(se, se_o) <= 2 ** -22


def test_noalloc_checks_heritabilities_before_writing(gw):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    P = make_problem(96, 40, 6, seed=36)
    lam, XLt, Xt, Yt, h2 = rotated_inputs(P, dev)
    for bad, code in ((1.5, gw.GWAS_ERR_ARG), (-0.2, gw.GWAS_ERR_ARG), (float("nan"), gw.GWAS_ERR_ARG)):
        hb = h2.clone()
        hb[3] = bad
        out = torch.full((2, P.t, P.m), float("nan"), dtype=torch.float32, device=dev)
        with pytest.raises(gw.GwasError) as e:
            gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lam, XLt, Xt, P.m, Yt, hb, P.t, gw.GWAS_OUT_LAST_SE, out)
        assert e.value.code == code
        assert torch.isnan(out).all()  # nothing was written
    # h2 = 1 with a zero eigenvalue: D_j has a zero entry, M_j is singular
    lz = lam.clone()
    lz[0] = 0.0
    h1 = torch.ones_like(h2)
    out = torch.full((2, P.t, P.m), float("nan"), dtype=torch.float32, device=dev)
    with pytest.raises(gw.GwasError) as e:
        gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lz, XLt, Xt, P.m, Yt, h1, P.t, gw.GWAS_OUT_LAST_SE, out)
    assert e.value.code == gw.GWAS_ERR_NOT_SPD


def test_noalloc_refuses_memory_kernels_cannot_use(gw):
    """Host arrays are refused: by the binding (numpy, CPU tensors), and by the C entry point
    itself when it is handed a page-locked host pointer, before any device work."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    P = make_problem(64, 20, 4, seed=37)
    lam, XLt, Xt, Yt, h2 = rotated_inputs(P, dev)
    out = torch.empty((2, P.t, P.m), dtype=torch.float32, device=dev)
    with pytest.raises(TypeError):
        gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lam.cpu().numpy(), XLt, Xt, P.m, Yt, h2, P.t, gw.GWAS_OUT_LAST_SE, out)
    with pytest.raises(ValueError):  # an output smaller than t * m pairs
        gw.gwas_solve_fp64_noalloc(P.n, P.pm1, lam, XLt, Xt, P.m, Yt, h2, P.t, gw.GWAS_OUT_LAST_SE, out[:, :, :-1])
    pinned = Yt.cpu().pin_memory()
    sing = ctypes.c_int64(0)
    rc = gw.lib.gwas_solve_fp64_noalloc(P.n, P.pm1, lam.data_ptr(), XLt.data_ptr(), Xt.data_ptr(), P.m,
                                        pinned.data_ptr(), h2.data_ptr(), P.t, gw.GWAS_OUT_LAST_SE, out.data_ptr(),
                                        None, ctypes.byref(sing))
    assert rc == gw.GWAS_ERR_ARG


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
