"""The mixed path's per-pair solve divides by the Schur complement and takes a square root for the
SE with branch-free routines of its own (the hardware approximations, the reciprocal refined by one
Newton-Raphson step): checked on the GPU against CUDA's correctly rounded __frcp_rn and __fsqrt_rn
over 36 orders of magnitude, both signs for the reciprocal."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_reciprocal_and_square_root_against_correctly_rounded(gw):
    rng = np.random.default_rng(7)
    mag = 10.0 ** rng.uniform(-18, 18, 200_000)
    special = np.array([1, 2, 3, 0.1, 0.5, 7, 1e-6, 1e6, 1000.0, 999.0, 2 ** -20, 2 ** 20], np.float64)
    x = np.concatenate([mag, special]).astype(np.float32)
    x = np.concatenate([x, -x])
    r = gw.gwas_check_epilogue_math(x)
    # reciprocal: within one ulp of the correctly rounded value (same sign, so the bit patterns
    # differ by the ulp count)
    ulps = np.abs(r[:, 0].view(np.int32).astype(np.int64) - r[:, 1].view(np.int32).astype(np.int64))
    assert np.all(np.isfinite(r[:, 0]))
    assert ulps.max() <= 1
    assert np.mean(ulps == 0) > 0.9          # nearly always the correctly rounded value itself
    # square root of the positive values: relative error within 2^-22
    pos = x > 0
    s, s_rn = r[pos, 2].astype(np.float64), r[pos, 3].astype(np.float64)
    assert np.max(np.abs(s - s_rn) / s_rn) <= 2.0 ** -22
