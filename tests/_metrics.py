"""Error metrics of the GPU results against the oracle.

Y is pure noise in the synthetic workloads, so true coefficients scatter
around zero and a pointwise relative error is unbounded.  The error of a pair
is therefore measured relative to max(|b*|, SE*): the coefficient's own size
or its standard error, whichever is larger.
"""
import numpy as np


def last_coef_err(beta, se, b_ref, se_ref):
    """max over pairs of |beta - beta*| / max(|beta*|, SE*) (SNP coefficient)."""
    bl = b_ref[..., -1]
    den = np.maximum(np.abs(bl), se_ref)
    return float(np.max(np.abs(beta - bl) / den))


def se_err(se, se_ref):
    return float(np.max(np.abs(se - se_ref) / se_ref))


def full_b_err(b, b_ref, se_ref):
    """max over pairs of ||b - b*||_inf / max(||b*||_inf, SE*)."""
    num = np.max(np.abs(b - b_ref), axis=-1)
    den = np.maximum(np.max(np.abs(b_ref), axis=-1), se_ref)
    return float(np.max(num / den))
