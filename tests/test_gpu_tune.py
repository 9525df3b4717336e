"""Autotuner of the fused kernel's launch shape and its JSON cache: a tuned context and a
context that reads the cache use the same shape and give the same results, a cached shape
other than the default is applied (the CTA pair), and an entry naming a shape that is not
built (another p, or a multi-CTA cluster other than the pair) is ignored."""
import json

import numpy as np
import pytest

from oracle import EigOracle
from synth import make_problem
from tests._metrics import last_coef_err, se_err

pytestmark = pytest.mark.gpu

DEFAULT = {"cs": 1, "ct": 1, "epw": 16, "pair": 0, "group": 16}


def solve(g, P, opts, tune=False):
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, opts)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        ms = g.gwas_autotune(ctx, P.Y, P.t, P.m) if tune else None
        shape = g.gwas_tune_shape(ctx)
        out = np.full((2, P.t, P.m), np.nan, dtype=np.float32)
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
        return out, shape, ms
    finally:
        g.gwas_destroy(ctx)


def check(out, b, se):
    beta, s = out[0].T.astype(np.float64), out[1].T.astype(np.float64)
    assert last_coef_err(beta, s, b, se) <= 1e-6 and se_err(s, se) <= 1e-6


def test_autotune_writes_and_reads_the_cache(gw, tmp_path):
    P = make_problem(256, 1500, 70, seed=3030)
    cache = str(tmp_path / "tune.json")
    opts = lambda: gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE, tune_cache=cache)
    out1, shape1, ms = solve(gw, P, opts(), tune=True)
    assert ms > 0
    entries = json.load(open(cache))
    assert len(entries) == 1
    key, entry = next(iter(entries.items()))
    assert key == "n=256,p=4,mode=mixed,t=2^6"
    assert {k: entry[k] for k in DEFAULT} == shape1
    out2, shape2, _ = solve(gw, P, opts())
    assert shape2 == shape1
    np.testing.assert_array_equal(out2, out1)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check(out1, b, se)


def test_cached_pair_shape_is_applied(gw, tmp_path):
    P = make_problem(200, 900, 40, seed=3031)
    cache = tmp_path / "tune.json"
    pair = {"cs": 2, "ct": 1, "epw": 16, "pair": 1, "group": 8}
    cache.write_text(json.dumps({"n=200,p=4,mode=mixed,t=2^5": dict(pair, ms=1.0)}))
    opts = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE, tune_cache=str(cache))
    out, shape, _ = solve(gw, P, opts)
    assert shape == pair
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check(out, b, se)


def test_unbuilt_shape_in_the_cache_is_ignored(gw, tmp_path):
    P = make_problem(160, 300, 20, pm1=5, seed=3032)  # p = 6: only the one-CTA shape is built
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({"n=160,p=6,mode=mixed,t=2^4": {"cs": 2, "ct": 1, "epw": 16, "pair": 1, "group": 8}}))
    opts = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE, tune_cache=str(cache))
    out, shape, _ = solve(gw, P, opts)
    assert shape == DEFAULT
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    check(out, b, se)


def test_cluster_shapes_without_a_kernel_are_ignored(gw, tmp_path, monkeypatch):
    """Only the one-CTA shapes and the CTA pair are built: a cached or forced 1x2, 2x1 or 2x2
    cluster shape (no such kernel exists) leaves the default shape in place."""
    P = make_problem(192, 700, 36, seed=3034)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    for cs, ct in ((1, 2), (2, 1), (2, 2)):
        cache = tmp_path / f"tune_{cs}{ct}.json"
        cache.write_text(json.dumps({"n=192,p=4,mode=mixed,t=2^5": {"cs": cs, "ct": ct, "epw": 16, "pair": 0,
                                                                     "group": 8}}))
        opts = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE, tune_cache=str(cache))
        out, shape, _ = solve(gw, P, opts)
        assert shape == DEFAULT
        check(out, b, se)
    monkeypatch.setenv("GWAS_FUSED_SHAPE", "2x2x16")
    out, _, _ = solve(gw, P, gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE))
    check(out, b, se)


def test_autotune_states(gw):
    P = make_problem(128, 200, 8, seed=3033)
    o = gw.gwas_default_opts(precision=gw.GWAS_FP64, output=gw.GWAS_OUT_LAST_SE)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        gw.gwas_load_snps(ctx, P.m, P.XR, P.n)
        with pytest.raises(gw.GwasError) as e:   # the FP64 path has no launch shape
            gw.gwas_autotune(ctx, P.Y)
        assert e.value.code == gw.GWAS_ERR_UNSUPPORTED
    finally:
        gw.gwas_destroy(ctx)
    o = gw.gwas_default_opts(precision=gw.GWAS_MIXED, output=gw.GWAS_OUT_LAST_SE)
    ctx = gw.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        with pytest.raises(gw.GwasError) as e:   # nothing to time before the genotypes are loaded
            gw.gwas_autotune(ctx, P.Y)
        assert e.value.code == gw.GWAS_ERR_STATE
        assert gw.gwas_tune_shape(ctx) == DEFAULT
    finally:
        gw.gwas_destroy(ctx)
