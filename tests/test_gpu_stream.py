"""Output streaming: host outputs by trait block (double-buffered copies) and the
callback API give bit-identical results to a device output."""
import ctypes

import numpy as np
import pytest

from synth import make_problem

pytestmark = pytest.mark.gpu


def device_result(g, P, prec, output):
    import torch
    o = g.gwas_default_opts(precision=prec, output=output)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        shape = (P.t, P.m, P.p) if output == g.GWAS_OUT_FULL_B else (2, P.t, P.m)
        dt = torch.float64 if output == g.GWAS_OUT_FULL_B else torch.float32
        out = torch.empty(shape, dtype=dt, device="cuda")
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
        return out.cpu().numpy()
    finally:
        g.gwas_destroy(ctx)


@pytest.mark.parametrize("prec,output", [(1, 1), (1, 0), (0, 1)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_output_by_blocks(gw, prec, output, pinned):
    import torch
    P = make_problem(200, 300, 45, seed=17)
    ref = device_result(gw, P, prec, output)
    o = gw.gwas_default_opts(precision=prec, output=output, trait_block=13)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        dt = torch.float64 if output == gw.GWAS_OUT_FULL_B else torch.float32
        out = torch.full(ref.shape, float("nan"), dtype=dt)
        if pinned:
            out = out.pin_memory()
        gw.gwas_solve(ctx, P.Y, 0, P.m, out)
    finally:
        gw.gwas_destroy(ctx)
    np.testing.assert_array_equal(out.numpy(), ref)


@pytest.mark.parametrize("prec,output", [(1, 1), (0, 0)])
def test_stream_callback(gw, prec, output):
    import torch
    P = make_problem(160, 257, 70, seed=19)
    ref = device_result(gw, P, prec, output)
    o = gw.gwas_default_opts(precision=prec, output=output)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    blk, M = 16, 200
    i0, i1 = 31, 31 + M
    got = np.full(ref.shape[:-1] + (M,) if output == gw.GWAS_OUT_LAST_SE else (P.t, M, P.p), np.nan,
                  dtype=ref.dtype)
    per = blk * M * (2 if output == gw.GWAS_OUT_LAST_SE else P.p)
    dt = torch.float32 if output == gw.GWAS_OUT_LAST_SE else torch.float64
    bufs = [torch.empty(per, dtype=dt).pin_memory() for _ in range(2)]
    seen = []

    def on_block(j0, nb, ptr):
        n_el = nb * M * (2 if output == gw.GWAS_OUT_LAST_SE else P.p)
        ct = ctypes.c_float if output == gw.GWAS_OUT_LAST_SE else ctypes.c_double
        arr = np.ctypeslib.as_array((ct * n_el).from_address(ptr)).copy()
        if output == gw.GWAS_OUT_LAST_SE:
            arr = arr.reshape(2, nb, M)
            got[:, j0:j0 + nb] = arr
        else:
            got[j0:j0 + nb] = arr.reshape(nb, M, P.p)
        seen.append((j0, nb))

    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        gw.gwas_solve_stream(ctx, P.Y, i0, i1, blk, bufs[0], bufs[1], on_block)
    finally:
        gw.gwas_destroy(ctx)
    assert seen == [(j, min(blk, P.t - j)) for j in range(0, P.t, blk)]
    if output == gw.GWAS_OUT_LAST_SE:
        np.testing.assert_array_equal(got, ref[:, :, i0:i1])
    else:
        np.testing.assert_array_equal(got, ref[:, i0:i1])
