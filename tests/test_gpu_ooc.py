"""Out-of-core solve (gwas_solve_ooc): genotype slabs streamed from host memory give the
same results as gwas_load_snps + gwas_solve, bit for bit, on both precision paths, with a
ragged last slab, several trait blocks, and pageable, page-locked or device genotypes."""
import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem
from tests._metrics import full_b_err, last_coef_err, se_err

pytestmark = pytest.mark.gpu


def in_core(g, P, precision, output):
    o = g.gwas_default_opts(precision=precision, output=output)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        out = np.full((P.t, P.m, P.p), np.nan) if output == g.GWAS_OUT_FULL_B else \
            np.full((2, P.t, P.m), np.nan, dtype=np.float32)
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
        return out
    finally:
        g.gwas_destroy(ctx)


def out_of_core(g, P, precision, output, slab, block, xr=None):
    o = g.gwas_default_opts(precision=precision, output=output)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    full_b = output == g.GWAS_OUT_FULL_B
    rows = min((slab or 1 << 20) + 127, P.m + 127) // 128 * 128   # the slab the library uses
    if full_b:
        out = np.full((P.t, P.m, P.p), np.nan)
        bufs = [np.empty(rows * block * P.p), np.empty(rows * block * P.p)]
    else:
        out = np.full((2, P.t, P.m), np.nan, dtype=np.float32)
        bufs = [np.empty(2 * rows * block, np.float32), np.empty(2 * rows * block, np.float32)]
    seen = []

    def piece(i0, i1, j0, nb, ptr):
        buf = bufs[0] if ptr == bufs[0].ctypes.data else bufs[1]
        assert ptr == buf.ctypes.data
        M = i1 - i0
        seen.append((i0, i1, j0, nb))
        if full_b:
            out[j0:j0 + nb, i0:i1] = buf[:nb * M * P.p].reshape(nb, M, P.p)
        else:
            out[:, j0:j0 + nb, i0:i1] = buf[:2 * nb * M].reshape(2, nb, M)

    try:
        XR = P.XR if xr is None else xr
        g.gwas_solve_ooc(ctx, P.m, XR, slab, P.Y, block, bufs[0], bufs[1], piece, n=P.n)
    finally:
        g.gwas_destroy(ctx)
    return out, seen


@pytest.mark.parametrize("precision_name,pm1", [("GWAS_MIXED", 3), ("GWAS_MIXED", 5), ("GWAS_MIXED", 11),
                                                 ("GWAS_FP64", 2), ("GWAS_FP64", 15)])
@pytest.mark.parametrize("output_name", ["GWAS_OUT_LAST_SE", "GWAS_OUT_FULL_B"])
def test_ooc_equals_in_core(gw, precision_name, pm1, output_name):
    precision, output = getattr(gw, precision_name), getattr(gw, output_name)
    P = make_problem(200, 1000, 40, pm1=pm1, seed=61 + pm1)
    ref = in_core(gw, P, precision, output)
    out, seen = out_of_core(gw, P, precision, output, slab=300, block=24)
    # slabs of 384 SNPs (300 rounded up to 128): [0,384) [384,768) [768,1000); trait blocks [0,24) [24,40)
    assert seen == [(0, 384, 0, 24), (0, 384, 24, 16), (384, 768, 0, 24), (384, 768, 24, 16),
                    (768, 1000, 0, 24), (768, 1000, 24, 16)]
    np.testing.assert_array_equal(out, ref)


def test_ooc_sources_and_oracle(gw):
    import torch
    P = make_problem(160, 700, 20, pm1=3, seed=71)
    ref = in_core(gw, P, gw.GWAS_MIXED, gw.GWAS_OUT_LAST_SE)
    pinned = torch.from_numpy(P.XR).pin_memory()
    on_dev = torch.from_numpy(P.XR).cuda()
    for xr in (pinned, on_dev):
        out, _ = out_of_core(gw, P, gw.GWAS_MIXED, gw.GWAS_OUT_LAST_SE, slab=256, block=20, xr=xr)
        np.testing.assert_array_equal(out, ref)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    beta, s = out[0].T.astype(np.float64), out[1].T.astype(np.float64)
    assert last_coef_err(beta, s, b, se) <= 1e-6 and se_err(s, se) <= 1e-6


def test_ooc_one_slab_and_state(gw):
    # one slab holding every SNP; afterwards the context holds no genotypes
    P = make_problem(128, 100, 3, seed=72)
    out, seen = out_of_core(gw, P, gw.GWAS_FP64, gw.GWAS_OUT_FULL_B, slab=0, block=8)
    assert seen == [(0, 100, 0, 3)]
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    assert full_b_err(out.transpose(1, 0, 2), b, se) <= 1e-10
