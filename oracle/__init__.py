"""CPU oracle for the multi-trait GWAS grid of GLS problems (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it.  It is a plain, slow, FP64
restatement of what the paper's method computes and shares no code with the
CUDA path.

* :func:`direct_gls` -- the definition, Eq. (1) with the covariance of Eq. (2),
  whitened by the Cholesky factor of each M_j (Section 3.1) and solved as a
  least-squares problem by QR.
* :class:`EigOracle` -- Algorithm 5 ("MT-GWAS") in GEMM form: one
  eigendecomposition of Phi, rotations by Z^T, per-trait quantities (D_j, K_j,
  W_L, v_j, S_TL, b_T) and per-pair quantities (W_R, S_BL, S_BR, b_B), then the
  p x p SPD solve by Cholesky.

Both return the coefficient vector b_ij (p entries, the SNP coefficient last)
and the standard error of the SNP coefficient.  The paper defines no standard
error; both functions use the textbook GLS one with the residual variance
estimated per pair: sigma^2 = RSS / (n - p), SE = sqrt(sigma^2 [S^-1]_pp),
where RSS is the squared norm of the whitened residual.
"""
from .gls import EigOracle, direct_gls, eig_gls  # noqa: F401
