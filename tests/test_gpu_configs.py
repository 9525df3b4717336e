"""Parity at the full sizes of the serving and paper-scale workloads, on sampled pairs that the
oracle computes one by one:

- serving: n = 2000, p = 4, 10^6 resident SNPs, a stream of requests with t_k log-uniform on
  [1, 2000] and SNP ranges log-uniform on [10^4, 10^6], all in flight together;
- paper scale: n = 1000, p = 4, m = 10^6, t = 10^5 (the shape of the paper's Section 4
  example), traits in blocks of 5000 whose SNP coefficient and SE stream to two page-locked host
  buffers through gwas_solve_stream.
"""
import ctypes

import numpy as np
import pytest

import bench
from oracle import EigOracle
from synth import BASE_SEED, covariates, genotypes, heritabilities, kinship, phenotypes, serving_requests
from tests._metrics import last_coef_err, se_err

pytestmark = pytest.mark.gpu

TOL = 1e-6


def check(beta, se_hat, b, se):
    assert last_coef_err(beta, se_hat, b, se) <= TOL and se_err(se_hat, se) <= TOL


def test_serving_at_full_size(gw):
    torch = pytest.importorskip("torch")
    n, m, pm1 = 2000, 1_000_000, 3
    dev = torch.device("cuda:0")
    phi, XL = kinship(n), covariates(n, pm1)
    XR = genotypes(n, m, BASE_SEED + 100)
    reqs = serving_requests(40, m, BASE_SEED + 1)
    rng = np.random.default_rng(BASE_SEED + 7)
    inputs = [(rng.standard_normal((r["t"], n)), rng.uniform(0.1, 0.9, r["t"])) for r in reqs]
    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
    ctx = gw.gwas_setup(n, pm1, phi, XL, 1, inputs[0][1][:1], o)
    samples = []
    try:
        gw.gwas_load_snps(ctx, m, torch.from_numpy(XR).to(dev), n)
        outs, ids = [], []
        for r, (Y, h2) in zip(reqs, inputs):   # all submitted at once: they share rounds
            out = torch.empty((2, r["t"], r["i1"] - r["i0"]), dtype=torch.float32, device=dev)
            outs.append(out)
            ids.append(gw.gwas_submit(ctx, Y, r["t"], h2, r["i0"], r["i1"], out))
        for rid in ids:
            assert gw.gwas_wait(ctx, rid, 600.0) == gw.GWAS_OK
        rounds, graph_rounds = gw.gwas_serve_stats(ctx)
        for r, out in zip(reqs, outs):
            M = r["i1"] - r["i0"]
            si = np.unique(np.concatenate([[0, M - 1], rng.choice(M, min(M, 30), replace=False)]))
            tj = np.unique(np.concatenate([[0, r["t"] - 1], rng.choice(r["t"], min(r["t"], 6), replace=False)]))
            got = out[:, torch.from_numpy(tj).to(dev)][:, :, torch.from_numpy(si).to(dev)].cpu().numpy()
            samples.append((r, si, tj, got, bool(torch.isfinite(out).all().item())))
    finally:
        gw.gwas_destroy(ctx)
    assert graph_rounds >= 1 and graph_rounds == rounds - 1
    oracle = EigOracle(phi, XL)
    for (r, si, tj, got, finite), (Y, h2) in zip(samples, inputs):
        assert finite
        b, se = oracle.solve(XR[r["i0"] + si], Y[tj], h2[tj])
        check(got[0].T.astype(np.float64), got[1].T.astype(np.float64), b, se)


def test_paper_scale_streamed_to_host(gw):
    torch = pytest.importorskip("torch")
    n, m, t, pm1, block = 1000, 1_000_000, 100_000, 3, 5000
    dev = torch.device("cuda:0")
    phi, XL, h2 = kinship(n), covariates(n, pm1), heritabilities(t)
    XR = genotypes(n, m)
    Y = phenotypes(n, t)
    rng = np.random.default_rng(2)
    si = np.unique(np.concatenate([np.arange(32), m - 32 + np.arange(32), rng.choice(m, 192, replace=False)]))
    tj = np.unique(np.concatenate([np.arange(8), t - 8 + np.arange(8), rng.choice(t, 112, replace=False)]))
    per = 2 * block * m
    bufs = [bench.pinned_host_array((per,), np.float32, torch)[0] for _ in range(2)]
    assert all(b is not None for b in bufs)
    got = np.full((2, tj.size, si.size), np.nan, np.float32)
    seen, nonfinite = [], []

    def on_block(j0, nb, ptr):
        blk = np.ctypeslib.as_array((ctypes.c_float * (2 * nb * m)).from_address(ptr)).reshape(2, nb, m)
        sel = np.nonzero((tj >= j0) & (tj < j0 + nb))[0]
        got[:, sel] = blk[:, (tj[sel] - j0)[:, None], si[None, :]]
        nonfinite.append(int((~np.isfinite(blk[:, ::97, ::101])).sum()))  # a strided sample of the block
        seen.append((j0, nb))

    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
    ctx = gw.gwas_setup(n, pm1, phi, XL, t, h2, o)
    try:
        gw.gwas_load_snps(ctx, m, torch.from_numpy(XR).to(dev), n)
        rc = gw.gwas_solve_stream(ctx, torch.from_numpy(Y).to(dev), 0, m, block, bufs[0], bufs[1], on_block)
        assert rc == gw.GWAS_OK
    finally:
        gw.gwas_destroy(ctx)
        for b in bufs:
            if isinstance(b, np.ndarray):
                torch.cuda.cudart().cudaHostUnregister(b.ctypes.data)
    assert seen == [(j, block) for j in range(0, t, block)]
    assert sum(nonfinite) == 0
    b, se = EigOracle(phi, XL).solve(XR[si], Y[tj], h2[tj])
    check(got[0].T.astype(np.float64), got[1].T.astype(np.float64), b, se)
