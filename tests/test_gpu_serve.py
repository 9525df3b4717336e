"""Serving with continuous batching: every request's result is the same alone and in a
mix (bitwise: the arithmetic of a pair does not depend on its round, nor on whether the
round was launched directly or replayed from its captured CUDA graph), the same as a
separate gwas_solve of the request with S_BR contracted per pair as serving does
(GWAS_S_BR=exact), and within the parity bar of the oracle."""
import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem
from tests._metrics import last_coef_err, se_err

pytestmark = pytest.mark.gpu


def requests(P, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        tk = int(rng.integers(1, 90))
        ln = int(rng.integers(1, P.m))
        i0 = int(rng.integers(0, P.m - ln + 1))
        Y = rng.standard_normal((tk, P.n))
        h2 = rng.uniform(0.1, 0.9, tk)
        out.append((Y, h2, i0, i0 + ln))
    return out


def new_ctx(g, P, t=1, h2=None):
    o = g.gwas_default_opts(precision=g.GWAS_MIXED, output=g.GWAS_OUT_LAST_SE)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, t, P.h2[:t] if h2 is None else h2, o)
    g.gwas_load_snps(ctx, P.m, P.XR, P.n)
    return ctx


def alloc_out(tk, M, k):
    import torch
    t = torch.full((2, tk, M), float("nan"), dtype=torch.float32)
    return t.pin_memory() if k % 2 == 0 else t.cuda()


def test_alone_equals_mix_equals_solve(gw, monkeypatch):
    P = make_problem(256, 3000, 4, seed=41)
    reqs = requests(P, 14, 7)
    ctx = new_ctx(gw, P)
    try:
        alone = []
        for k, (Y, h2, i0, i1) in enumerate(reqs):
            out = alloc_out(len(h2), i1 - i0, k)
            rid = gw.gwas_submit(ctx, Y, len(h2), h2, i0, i1, out)
            assert gw.gwas_wait(ctx, rid, 120.0) == gw.GWAS_OK
            alone.append(out.cpu().numpy())
        outs, ids = [], []
        for k, (Y, h2, i0, i1) in enumerate(reqs):      # all at once: they share rounds
            out = alloc_out(len(h2), i1 - i0, k + 1)
            outs.append(out)
            ids.append(gw.gwas_submit(ctx, Y, len(h2), h2, i0, i1, out))
        for rid in ids:
            assert gw.gwas_wait(ctx, rid, 120.0) == gw.GWAS_OK
        mix = [o.cpu().numpy() for o in outs]
        ts = [gw.gwas_request_times(ctx, rid) for rid in ids]
        rounds, graph_rounds = gw.gwas_serve_stats(ctx)
    finally:
        gw.gwas_destroy(ctx)
    # the first round launches directly and is captured; the others replay the CUDA graph
    assert rounds >= len(reqs) + 1 and graph_rounds == rounds - 1
    for a, b in zip(alone, mix):
        np.testing.assert_array_equal(a, b)
    assert all(t0 <= t1 <= t2 for t0, t1, t2 in ts)
    # the same request through gwas_solve, and the oracle on a sample of requests
    monkeypatch.setenv("GWAS_S_BR", "exact")
    for k in (0, 3, 9):
        Y, h2, i0, i1 = reqs[k]
        ctx = new_ctx(gw, P, t=len(h2), h2=h2)
        try:
            out = np.empty((2, len(h2), i1 - i0), np.float32)
            gw.gwas_solve(ctx, Y, i0, i1, out)
        finally:
            gw.gwas_destroy(ctx)
        np.testing.assert_array_equal(out, alone[k])
        b, se = EigOracle(P.phi, P.XL).solve(P.XR[i0:i1], Y, h2)
        assert last_coef_err(out[0].T.astype(np.float64), out[1].T.astype(np.float64), b, se) <= 1e-6
        assert se_err(out[1].T.astype(np.float64), se) <= 1e-6


def test_poll_and_singular_request(gw):
    P = make_problem(128, 700, 2, seed=42)
    P.XR[300] = 0
    ctx = new_ctx(gw, P)
    try:
        rng = np.random.default_rng(3)
        Y = rng.standard_normal((40, P.n))
        h2 = rng.uniform(0.1, 0.9, 40)
        out = alloc_out(40, 400, 1)
        rid = gw.gwas_submit(ctx, Y, 40, h2, 100, 500, out)
        assert gw.gwas_wait(ctx, rid, 120.0) == gw.GWAS_ERR_SINGULAR_PAIRS
        done, rc = gw.gwas_poll(ctx, rid)
        assert done and rc == gw.GWAS_ERR_SINGULAR_PAIRS
        o = out.cpu().numpy()
        assert np.isnan(o[:, :, 200]).all() and np.isfinite(np.delete(o, 200, axis=2)).all()
        with pytest.raises(gw.GwasError):
            gw.gwas_submit(ctx, Y, 40, h2, 0, 10, np.empty((2, 40, 10), np.float32))  # pageable output
    finally:
        gw.gwas_destroy(ctx)


@pytest.mark.parametrize("pm1", [0, 5, 9, 14])
def test_serving_general_p(gw, pm1, monkeypatch):
    """Serving with q = p - 1 other than 3 (tiles of 16 traits for q = 5 and 9, of 8 for
    q = 14): a mix of requests equals gwas_solve of each request and the oracle."""
    P = make_problem(160, 1200, 2, pm1=pm1, seed=43 + pm1)
    reqs = requests(P, 6, 11 + pm1)
    ctx = new_ctx(gw, P)
    try:
        outs, ids = [], []
        for k, (Y, h2, i0, i1) in enumerate(reqs):
            out = alloc_out(len(h2), i1 - i0, k)
            outs.append(out)
            ids.append(gw.gwas_submit(ctx, Y, len(h2), h2, i0, i1, out))
        for rid in ids:
            assert gw.gwas_wait(ctx, rid, 120.0) == gw.GWAS_OK
        mix = [o.cpu().numpy() for o in outs]
    finally:
        gw.gwas_destroy(ctx)
    monkeypatch.setenv("GWAS_S_BR", "exact")
    for k in (0, 2, 5):
        Y, h2, i0, i1 = reqs[k]
        ctx = new_ctx(gw, P, t=len(h2), h2=h2)
        try:
            out = np.empty((2, len(h2), i1 - i0), np.float32)
            gw.gwas_solve(ctx, Y, i0, i1, out)
        finally:
            gw.gwas_destroy(ctx)
        np.testing.assert_array_equal(out, mix[k])
        b, se = EigOracle(P.phi, P.XL).solve(P.XR[i0:i1], Y, h2)
        assert last_coef_err(out[0].T.astype(np.float64), out[1].T.astype(np.float64), b, se) <= 1e-6
        assert se_err(out[1].T.astype(np.float64), se) <= 1e-6
