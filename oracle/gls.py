"""FP64 CPU oracle (test infrastructure; see the package docstring).

Layouts follow the C interface: ``XR`` is (m, n) (row i = SNP i), ``Y`` is
(t, n) (row j = trait j), ``XL`` is (p-1, n) (row l = covariate l).  Outputs:
``b`` of shape (m, t, p) with the SNP coefficient last, ``se`` of shape (m, t).

Parity of both functions is pinned by tests/test_oracle_pins.py (definition on
rational inputs, OLS at h^2 = 0 and at Phi = I, planted coefficients, the
normal-equation residual, invariances and the p = 1 closed form).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _covariance(phi: np.ndarray, h2: float, sigma2: float = 1.0) -> np.ndarray:
    """M_j = sigma_j^2 (h_j^2 Phi + (1 - h_j^2) I), Eq. (2)."""
    n = phi.shape[0]
    return sigma2 * (h2 * phi + (1.0 - h2) * np.eye(n))


def direct_gls(phi, XL, XR, Y, h2, sigma2=None):
    """b_ij = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j, Eq. (1), for every (i, j).

    For each trait j the covariance M_j of Eq. (2) is factored as L L^T
    (Section 3.1, the single-instance approach); the whitened problem
    L^-1 y_j ~ L^-1 X_i is an ordinary least-squares problem, solved by a QR
    factorisation of the whitened design.  Cost O(t n^3 + t m n^2): small
    inputs only.
    """
    XL = np.asarray(XL, dtype=np.float64).reshape(-1, np.shape(phi)[0])
    XR = np.asarray(XR, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = phi.shape[0]
    pm1 = XL.shape[0]
    p = pm1 + 1
    m, t = XR.shape[0], Y.shape[0]
    sig = np.ones(t) if sigma2 is None else np.asarray(sigma2, dtype=np.float64)
    b = np.empty((m, t, p))
    se = np.empty((m, t))
    for j in range(t):
        L = np.linalg.cholesky(_covariance(phi, h2[j], sig[j]))
        wl = sla.solve_triangular(L, XL.T, lower=True)          # n x (p-1)
        wr = sla.solve_triangular(L, XR.T, lower=True)          # n x m
        v = sla.solve_triangular(L, Y[j], lower=True)           # n
        X = np.empty((m, n, p))                                 # whitened X_i, stacked over i
        X[:, :, :pm1] = wl[None, :, :]
        X[:, :, pm1] = wr.T
        Q, R = np.linalg.qr(X)                                  # (m, n, p), (m, p, p)
        qv = np.einsum("mnp,n->mp", Q, v)
        bj = np.linalg.solve(R, qv[..., None])[..., 0]
        res = v[None, :] - np.einsum("mnp,mp->mn", X, bj)
        rss = np.einsum("mn,mn->m", res, res)
        rinv = np.linalg.inv(R)
        s_inv_pp = np.einsum("mk,mk->m", rinv[:, pm1, :], rinv[:, pm1, :])
        b[:, j, :] = bj
        se[:, j] = np.sqrt(rss / (n - p) * s_inv_pp)
    return b, se


def _chol_solve_batched(S: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Solve S x = c for a stack of SPD p x p systems by Cholesky (LAPACK posv)."""
    L = np.linalg.cholesky(S)
    p = S.shape[-1]
    z = np.empty_like(c)
    for r in range(p):                       # forward substitution, L z = c
        z[..., r] = (c[..., r] - np.einsum("...k,...k->...", L[..., r, :r], z[..., :r])) / L[..., r, r]
    x = np.empty_like(c)
    for r in range(p - 1, -1, -1):           # back substitution, L^T x = z
        x[..., r] = (z[..., r] - np.einsum("...k,...k->...", L[..., r + 1:, r], x[..., r + 1:])) / L[..., r, r]
    return x


class EigOracle:
    """Algorithm 5 (MT-GWAS) in GEMM form, in FP64.

    Construction performs the preloop operations that do not involve the
    streams: the eigendecomposition Z Lambda Z^T = Phi and X'_L = Z^T X_L.
    :meth:`solve` then performs, for the given SNPs and traits, the rotations
    X'_R = Z^T X_R and Y' = Z^T Y and the double loop (traits outer, SNPs
    vectorised), with the paper's K_j = D_j^(-1/2) and W = K_j^T X'.
    """

    def __init__(self, phi, XL):
        phi = np.asarray(phi, dtype=np.float64)
        self.n = phi.shape[0]
        self.XL = np.asarray(XL, dtype=np.float64).reshape(-1, self.n)
        self.pm1 = self.XL.shape[0]
        lam, Z = np.linalg.eigh(phi)           # Z Lambda Z^T = Phi (eigendec)
        self.lam, self.Z = lam, Z
        self.XLr = Z.T @ self.XL.T             # X'_L := Z^T X_L (gemm), n x (p-1)

    def solve(self, XR, Y, h2, sigma2=None):
        n, pm1 = self.n, self.pm1
        p = pm1 + 1
        XR = np.asarray(XR, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        m, t = XR.shape[0], Y.shape[0]
        sig = np.ones(t) if sigma2 is None else np.asarray(sigma2, dtype=np.float64)
        XRr = self.Z.T @ XR.T                  # X'_R := Z^T X_R (gemm), n x m
        Yr = self.Z.T @ Y.T                    # Y' := Z^T Y (gemm), n x t
        b = np.empty((m, t, p))
        se = np.empty((m, t))
        for j in range(t):
            D = sig[j] * (h2[j] * self.lam + (1.0 - h2[j]))   # D_j
            K = 1.0 / np.sqrt(D)                                # K_j = D_j^(-1/2)
            WL = K[:, None] * self.XLr                          # W_Lj := K_j^T X'_L
            v = K * Yr[:, j]                                    # v_j := K_j^T y'_j
            S_TL = WL.T @ WL                                    # syrk
            b_T = WL.T @ v                                      # gemv
            WR = K[:, None] * XRr                               # W_Rij := K_j^T X'_Ri, all i
            S_BL = WR.T @ WL                                    # m x (p-1)
            S_BR = np.einsum("ki,ki->i", WR, WR)                # m
            b_B = WR.T @ v                                      # m
            S = np.empty((m, p, p))
            S[:, :pm1, :pm1] = S_TL
            S[:, pm1, :pm1] = S_BL
            S[:, :pm1, pm1] = S_BL
            S[:, pm1, pm1] = S_BR
            c = np.empty((m, p))
            c[:, :pm1] = b_T
            c[:, pm1] = b_B
            bj = _chol_solve_batched(S, c)                      # posv
            res = v[:, None] - WL @ bj[:, :pm1].T - WR * bj[:, pm1][None, :]
            rss = np.einsum("ki,ki->i", res, res)
            ep = np.zeros((m, p))
            ep[:, pm1] = 1.0
            s_inv_pp = _chol_solve_batched(S, ep)[:, pm1]
            b[:, j, :] = bj
            se[:, j] = np.sqrt(rss / (n - p) * s_inv_pp)
        return b, se


def eig_gls(phi, XL, XR, Y, h2, sigma2=None):
    """One-shot :class:`EigOracle` (eigendecomposition + solve)."""
    return EigOracle(phi, XL).solve(XR, Y, h2, sigma2)
