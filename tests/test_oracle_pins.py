"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* exact rational arithmetic of the definition (Eq. 1-2) on tiny inputs;
* the two oracle routes against each other (Cholesky/QR vs. Algorithm 5);
* OLS closed forms: h^2 = 0 and Phi = I (then M_j is a multiple of I);
* planted coefficients (noise-free y = X_i beta);
* the per-pair optimality certificate X_i^T M_j^-1 (y_j - X_i b_ij) = 0;
* invariances: sigma_j^2 scaling (Eq. 2), eigenvector signs, linearity in y;
* the p = 1 closed form b = x^T M^-1 y / x^T M^-1 x;
* planted mistakes in the oracle are caught by these pins.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import oracle.gls as og
from oracle import EigOracle, direct_gls, eig_gls
from synth import make_problem

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def small():
    return make_problem(96, 40, 6, pm1=3, seed=7)


@pytest.fixture(scope="module")
def wide():
    # p = 20, the top of the paper's range (Section 3)
    return make_problem(96, 24, 4, pm1=19, seed=8)


both_p = pytest.mark.parametrize("case", ["small", "wide"])


# ---------------------------------------------------------------- rational
def _frac_solve(A, B):
    """Gauss-Jordan elimination over the rationals: A^-1 B."""
    n = len(A)
    M = [list(A[r]) + list(B[r]) for r in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


def _exact_gls(phi, X, y, h2):
    n, p = len(X), len(X[0])
    M = [[h2 * phi[r][c] + ((1 - h2) if r == c else 0) for c in range(n)] for r in range(n)]
    Minv_X = _frac_solve(M, X)
    Minv_y = _frac_solve(M, [[v] for v in y])
    S = [[sum(X[k][a] * Minv_X[k][b] for k in range(n)) for b in range(p)] for a in range(p)]
    c = [[sum(X[k][a] * Minv_y[k][0] for k in range(n))] for a in range(p)]
    b = [v[0] for v in _frac_solve(S, c)]
    r = [y[k] - sum(X[k][a] * b[a] for a in range(p)) for k in range(n)]
    Minv_r = _frac_solve(M, [[v] for v in r])
    rss = sum(r[k] * Minv_r[k][0] for k in range(n))
    e_p = [[Fraction(int(a == p - 1))] for a in range(p)]
    sinv_pp = _frac_solve(S, e_p)[p - 1][0]
    return b, rss / (n - p) * sinv_pp  # coefficients and SE^2


def test_rational_definition():
    rng = np.random.default_rng(3)
    n, pm1, m, t = 6, 2, 3, 2
    G = rng.integers(-2, 3, size=(n, 8))
    phi_i = G @ G.T + np.eye(n, dtype=np.int64)          # integer SPD
    phi = [[Fraction(int(v)) for v in row] for row in phi_i]
    XL = np.stack([np.ones(n), rng.integers(-3, 4, n)]).astype(np.int64)
    XR = rng.integers(0, 3, size=(m, n))
    Y = rng.integers(-5, 6, size=(t, n))
    h2 = [Fraction(1, 3), Fraction(7, 10)]
    bd, sd = direct_gls(phi_i.astype(float), XL.astype(float), XR, Y.astype(float), np.array([float(h) for h in h2]))
    be, se = eig_gls(phi_i.astype(float), XL.astype(float), XR, Y.astype(float), np.array([float(h) for h in h2]))
    for i in range(m):
        for j in range(t):
            X = [[Fraction(int(XL[0, k])), Fraction(int(XL[1, k])), Fraction(int(XR[i, k]))] for k in range(n)]
            b, se2 = _exact_gls(phi, X, [Fraction(int(v)) for v in Y[j]], h2[j])
            bx = np.array([float(v) for v in b])
            assert np.abs(bd[i, j] - bx).max() <= 1e-12 * max(1.0, np.abs(bx).max())
            assert np.abs(be[i, j] - bx).max() <= 1e-12 * max(1.0, np.abs(bx).max())
            assert abs(sd[i, j] ** 2 - float(se2)) <= 1e-12 * max(1.0, float(se2))
            assert abs(se[i, j] ** 2 - float(se2)) <= 1e-12 * max(1.0, float(se2))


# ---------------------------------------------------------------- two routes
@both_p
def test_eig_matches_direct(case, request):
    P = request.getfixturevalue(case)
    bd, sd = direct_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
    be, se = eig_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
    assert _rel(be, bd) < 1e-10
    assert _rel(se, sd) < 1e-10


def test_eig_matches_direct_tiny_config():
    # the smallest workload: n=256, p=4 (a slice of its SNPs and all 10 traits)
    P = make_problem(256, 64, 10)
    bd, sd = direct_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
    be, se = eig_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
    assert _rel(be, bd) < 1e-10 and _rel(se, sd) < 1e-10


# ---------------------------------------------------------------- OLS closed forms
def _ols(XL, xr, y):
    X = np.column_stack([XL.T, xr.astype(float)])
    b, res, rank, _ = np.linalg.lstsq(X, y, rcond=None)
    n, p = X.shape
    r = y - X @ b
    s2 = r @ r / (n - p)
    _, R = np.linalg.qr(X)
    Rinv = sla.solve_triangular(R, np.eye(p))
    return b, np.sqrt(s2 * (Rinv[p - 1] @ Rinv[p - 1]))


@both_p
@pytest.mark.parametrize("route", ["direct", "eig"])
def test_ols_at_h2_zero(case, route, request):
    P = request.getfixturevalue(case)
    h2 = np.zeros(P.t)
    f = direct_gls if route == "direct" else eig_gls
    b, se = f(P.phi, P.XL, P.XR, P.Y, h2)
    for i in range(0, P.m, 7):
        for j in range(P.t):
            bo, so = _ols(P.XL, P.XR[i], P.Y[j])
            assert np.abs(b[i, j] - bo).max() < 1e-10 * max(1, np.abs(bo).max())
            assert abs(se[i, j] - so) < 1e-10 * so


def test_ols_at_identity_kinship(small):
    P = small
    b, se = eig_gls(np.eye(P.n), P.XL, P.XR, P.Y, P.h2)
    for i in range(0, P.m, 5):
        for j in range(P.t):
            bo, so = _ols(P.XL, P.XR[i], P.Y[j])
            assert np.abs(b[i, j] - bo).max() < 1e-10 * max(1, np.abs(bo).max())
            assert abs(se[i, j] - so) < 1e-10 * so


# ---------------------------------------------------------------- planted coefficients
@both_p
def test_planted_coefficients(case, request):
    P = request.getfixturevalue(case)
    rng = np.random.default_rng(11)
    i = 5
    beta = rng.standard_normal(P.p)
    X = np.column_stack([P.XL.T, P.XR[i].astype(float)])
    Y = np.tile(X @ beta, (P.t, 1))
    for f in (direct_gls, eig_gls):
        b, se = f(P.phi, P.XL, P.XR[i:i + 1], Y, P.h2)
        assert np.abs(b[0] - beta[None, :]).max() < 1e-10
        assert se.max() < 1e-6


# ---------------------------------------------------------------- optimality certificate
@both_p
def test_normal_equation_residual(case, request):
    P = request.getfixturevalue(case)
    b, _ = eig_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
    for j in range(P.t):
        M = P.h2[j] * P.phi + (1 - P.h2[j]) * np.eye(P.n)
        cf = sla.cho_factor(M)
        for i in range(P.m):
            X = np.column_stack([P.XL.T, P.XR[i].astype(float)])
            g = X.T @ sla.cho_solve(cf, P.Y[j] - X @ b[i, j])
            ref = X.T @ sla.cho_solve(cf, P.Y[j])
            assert np.linalg.norm(g) <= 1e-12 * np.linalg.norm(ref)


# ---------------------------------------------------------------- invariances
def test_sigma_scaling_invariance(small):
    P = small
    sig = np.linspace(0.2, 5.0, P.t)
    b0, s0 = eig_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
    b1, s1 = eig_gls(P.phi, P.XL, P.XR, P.Y, P.h2, sigma2=sig)
    b2, s2 = direct_gls(P.phi, P.XL, P.XR[:6], P.Y, P.h2, sigma2=sig)
    assert _rel(b1, b0) < 1e-12 and _rel(s1, s0) < 1e-12
    assert _rel(b2, b0[:6]) < 1e-10 and _rel(s2, s0[:6]) < 1e-10


def test_eigenvector_sign_invariance(small):
    P = small
    o = EigOracle(P.phi, P.XL)
    b0, s0 = o.solve(P.XR, P.Y, P.h2)
    flip = np.where(np.arange(P.n) % 3 == 0, -1.0, 1.0)
    o.Z = o.Z * flip[None, :]
    o.XLr = o.Z.T @ o.XL.T
    b1, s1 = o.solve(P.XR, P.Y, P.h2)
    assert _rel(b1, b0) < 1e-12 and _rel(s1, s0) < 1e-12


def test_linearity_in_y(small):
    P = small
    o = EigOracle(P.phi, P.XL)
    y1, y2 = P.Y[:3], P.Y[3:6]
    b1, _ = o.solve(P.XR, y1, P.h2[:3])
    b2, _ = o.solve(P.XR, y2, P.h2[:3])
    b3, _ = o.solve(P.XR, y1 + 2.5 * y2, P.h2[:3])
    assert _rel(b3, b1 + 2.5 * b2) < 1e-11


# ---------------------------------------------------------------- p = 1
def test_single_column_closed_form(small):
    P = small
    XL = np.empty((0, P.n))
    b, se = eig_gls(P.phi, XL, P.XR, P.Y, P.h2)
    bd, sd = direct_gls(P.phi, XL, P.XR, P.Y, P.h2)
    for j in range(P.t):
        M = P.h2[j] * P.phi + (1 - P.h2[j]) * np.eye(P.n)
        Minv_y = np.linalg.solve(M, P.Y[j])
        Minv_X = np.linalg.solve(M, P.XR.T.astype(float))
        num = P.XR.astype(float) @ Minv_y
        den = np.einsum("ik,ki->i", P.XR.astype(float), Minv_X)
        assert np.abs(b[:, j, 0] - num / den).max() < 1e-10 * np.abs(num / den).max()
        assert np.abs(bd[:, j, 0] - num / den).max() < 1e-10 * np.abs(num / den).max()
    assert _rel(se, sd) < 1e-10


# ---------------------------------------------------------------- planted mistakes
class _NoSqrt:
    """numpy stand-in whose sqrt is the identity (drops the square root of K_j)."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def sqrt(x):
        return np.asarray(x)


def _pins_pass(P):
    try:
        bd, sd = direct_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
        be, se = eig_gls(P.phi, P.XL, P.XR, P.Y, P.h2)
        if not (_rel(be, bd) < 1e-10 and _rel(se, sd) < 1e-10):
            return False
        b0, s0 = eig_gls(P.phi, P.XL, P.XR, P.Y, np.zeros(P.t))
        for i in range(0, P.m, 9):
            for j in range(P.t):
                bo, so = _ols(P.XL, P.XR[i], P.Y[j])
                if np.abs(b0[i, j] - bo).max() > 1e-10 * max(1, np.abs(bo).max()):
                    return False
                if abs(s0[i, j] - so) > 1e-10 * so:
                    return False
        return True
    except Exception:
        return False


@pytest.mark.parametrize("mutation", ["drop_sqrt", "swap_h2", "skip_back_substitution", "sign_S_BL"])
def test_planted_mistakes_are_caught(small, monkeypatch, mutation):
    P = make_problem(48, 20, 4, pm1=3, seed=5)
    assert _pins_pass(P)
    if mutation == "drop_sqrt":
        monkeypatch.setattr(og, "np", _NoSqrt())
    elif mutation == "swap_h2":
        monkeypatch.setattr(og, "_covariance", lambda phi, h2, s=1.0: s * ((1 - h2) * phi + h2 * np.eye(phi.shape[0])))
    elif mutation == "skip_back_substitution":
        real = og._chol_solve_batched

        def broken(S, c):
            L = np.linalg.cholesky(S)
            return np.linalg.solve(L, c[..., None])[..., 0]
        monkeypatch.setattr(og, "_chol_solve_batched", broken)
        assert real is not broken
    elif mutation == "sign_S_BL":
        real_solve = og._chol_solve_batched

        def flipped(S, c):
            S = S.copy()
            S[:, -1, :-1] *= -1
            S[:, :-1, -1] *= -1
            return real_solve(S, c)
        monkeypatch.setattr(og, "_chol_solve_batched", flipped)
    assert not _pins_pass(P)
    assert oracle.EigOracle is EigOracle
