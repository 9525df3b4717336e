"""The planning rule of the interpolated S_BR (gwas_cheb_plan, host code: runs without a GPU).

For a SNP, S_BR(h) = sum_k y_k / (1 - h + h lambda_k) with y_k >= 0.  The library replaces it by
its interpolant at the R Chebyshev points of [lo, hi] and claims a relative error bound per term.
Here the interpolant is built independently (numpy polynomial fit through the nodes) and its
relative error is measured on a fine grid: it must stay under the bound the library reports,
the bound must meet the tolerance, and R must be the least number of nodes that meets it.
"""
import numpy as np
import pytest

from synth import covariates, kinship

def reachable_spectrum(n, pm1, seed=20121029):
    phi = kinship(n, seed)
    lam, Z = np.linalg.eigh(phi)
    if pm1 == 0:
        return lam, np.ones(n, bool)
    X = covariates(n, pm1, seed).T
    Pc = np.eye(n) - X @ np.linalg.solve(X.T @ X, X.T)
    rk = np.sum((Pc @ Z) ** 2, axis=0)
    return lam, rk > 1e-16


def measured_error(lam, reach, lo, hi, R):
    """max over reached k and a fine grid of h of |p_k(h) - f_k(h)| / f_k(h), p_k the interpolant
    of f_k(h) = 1 / (1 - h + h lambda_k) at the Chebyshev points of [lo, hi]."""
    r = np.arange(R)
    nodes = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.pi * r / (R - 1))
    h = np.linspace(lo, hi, 2001)
    # barycentric form (second kind) of the interpolant, evaluated away from the nodes
    w = (-1.0) ** r
    w[0] *= 0.5
    w[-1] *= 0.5
    d = h[:, None] - nodes[None, :]
    on = np.isclose(d, 0.0, atol=1e-15).any(axis=1)
    h, d = h[~on], d[~on]
    worst = 0.0
    for lk in np.unique(lam[reach]):
        f_nodes = 1.0 / (1.0 - nodes + nodes * lk)
        p = (w / d) @ f_nodes / np.sum(w / d, axis=1)
        f = 1.0 / (1.0 - h + h * lk)
        worst = max(worst, float(np.max(np.abs(p - f) / f)))
    return worst


@pytest.mark.parametrize("lo,hi", [(0.1, 0.9), (0.0, 1.0), (0.3, 0.31)])
def test_bound_holds_and_r_is_least(gw_cpu, lo, hi):
    lam, reach = reachable_spectrum(300, 3)
    R, bound = gw_cpu.gwas_cheb_plan(lam, reach, lo, hi, tol=1e-10)
    assert 4 <= R <= 24
    assert bound <= 1e-10
    assert measured_error(lam, reach, lo, hi, R) <= bound * 1.000001 + 1e-15
    # the bound is not loose by much: the measured error is within a few hundred of it
    assert measured_error(lam, reach, lo, hi, R) >= bound / 300
    if R > 4:
        # one node fewer does not meet the tolerance, by measurement
        assert measured_error(lam, reach, lo, hi, R - 1) > 1e-10 / 300


def test_looser_tolerance_needs_fewer_nodes(gw_cpu):
    lam, reach = reachable_spectrum(300, 3)
    r_tight, _ = gw_cpu.gwas_cheb_plan(lam, reach, 0.0, 1.0, tol=1e-12)
    r_loose, _ = gw_cpu.gwas_cheb_plan(lam, reach, 0.0, 1.0, tol=1e-6)
    assert 0 < r_loose < r_tight


def test_pole_near_or_inside_the_interval_is_refused(gw_cpu):
    # no covariates: the intercept direction (eigenvalue 1e-3 of the synthetic kinship) is
    # reached, its pole 1/(1 - 1e-3) sits just above h = 1, so [0, 1] needs far more than 24 nodes
    lam, reach = reachable_spectrum(200, 0)
    R, bound = gw_cpu.gwas_cheb_plan(lam, reach, 0.0, 1.0)
    assert R == 0 and bound > 1e-10
    # a negative eigenvalue puts a pole inside [0, 1]
    lam2 = np.array([-0.5, 0.4, 1.3])
    R, bound = gw_cpu.gwas_cheb_plan(lam2, np.ones(3, bool), 0.0, 1.0)
    assert R == 0 and not np.isfinite(bound)
    # the same eigenvalue outside the reach of the SNPs does not matter
    R, _ = gw_cpu.gwas_cheb_plan(lam2, np.array([False, True, True]), 0.0, 1.0)
    assert R > 0


def test_plan_arguments_are_checked(gw_cpu):
    lam = np.array([0.5, 1.5])
    with pytest.raises(gw_cpu.GwasError):
        gw_cpu.gwas_cheb_plan(lam, np.ones(2, bool), 0.5, 0.5)
    with pytest.raises(gw_cpu.GwasError):
        gw_cpu.gwas_cheb_plan(lam, np.ones(2, bool), -0.1, 0.5)
    with pytest.raises(ValueError):
        gw_cpu.gwas_cheb_plan(lam, np.ones(3, bool), 0.1, 0.5)
