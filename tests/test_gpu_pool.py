"""The library's device memory pool: a context set up after another reuses the memory the first
gave back (no new reservation), results do not depend on where buffers come from (bitwise equal
to a process that allocates with cudaMalloc, GWAS_POOL=0), gwas_pool_trim gives unused memory
back, and the pool entry points reject a device that does not exist."""
import os
import subprocess
import sys

import numpy as np
import pytest

from synth import make_problem

pytestmark = pytest.mark.gpu

MIB = 1 << 20

_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1210_7683_gb300 as g
from synth import make_problem
P = make_problem(320, 3000, 50, seed=901)
o = g.gwas_default_opts(precision=g.GWAS_MIXED, output=g.GWAS_OUT_LAST_SE)
ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
g.gwas_load_snps(ctx, P.m, P.XR, P.n)
out = np.empty((2, P.t, P.m), np.float32)
g.gwas_solve(ctx, P.Y, 0, P.m, out)
g.gwas_destroy(ctx)
assert g.gwas_pool_info(0) == {"reserved": 0, "used": 0}
np.save(sys.argv[2], out)
"""


def _solve(g, P, info_during=None):
    o = g.gwas_default_opts(precision=g.GWAS_MIXED, output=g.GWAS_OUT_LAST_SE)
    ctx = g.gwas_setup(P.n, P.pm1, P.phi, P.XL, P.t, P.h2, o)
    try:
        g.gwas_load_snps(ctx, P.m, P.XR, P.n)
        out = np.empty((2, P.t, P.m), np.float32)
        g.gwas_solve(ctx, P.Y, 0, P.m, out)
        if info_during is not None:
            info_during.append(g.gwas_pool_info(0))
    finally:
        g.gwas_destroy(ctx)
    return out


def test_pool_reuses_memory_and_trims(gw):
    P = make_problem(320, 3000, 50, seed=901)
    base = gw.gwas_pool_info(0)
    during = []
    a = _solve(gw, P, during)
    after_a = gw.gwas_pool_info(0)
    # the context's buffers came from the pool and went back to it, which kept them
    assert during[0]["used"] > base["used"]
    assert after_a["used"] == base["used"]
    assert after_a["reserved"] >= during[0]["used"]
    b = _solve(gw, P)
    after_b = gw.gwas_pool_info(0)
    assert after_b["reserved"] <= after_a["reserved"] + 32 * MIB   # no new mapping for the same sizes
    assert np.array_equal(a, b)
    gw.gwas_pool_trim(0, 0)
    trimmed = gw.gwas_pool_info(0)
    assert trimmed["used"] == base["used"]
    assert trimmed["reserved"] <= trimmed["used"] + 32 * MIB
    # after a trim the next context maps its memory again and gets the same results
    assert np.array_equal(_solve(gw, P), a)


def test_pool_off_gives_identical_results(gw, tmp_path, root):
    P = make_problem(320, 3000, 50, seed=901)
    pooled = _solve(gw, P)
    env = dict(os.environ, GWAS_POOL="0")
    path = str(tmp_path / "out.npy")
    subprocess.run([sys.executable, "-c", _CHILD, root, path], env=env, check=True, timeout=600)
    assert np.array_equal(np.load(path), pooled)


def test_pool_rejects_missing_device(gw):
    for dev in (-1, 1 << 20):
        with pytest.raises(gw.GwasError) as e:
            gw.gwas_pool_info(dev)
        assert e.value.code == gw.GWAS_ERR_ARG
        with pytest.raises(gw.GwasError) as e:
            gw.gwas_pool_trim(dev, 0)
        assert e.value.code == gw.GWAS_ERR_ARG
