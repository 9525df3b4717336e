// Eigendecomposition of the kinship matrix, Phi = Z Lambda Z^T (the preloop of Algorithm 5):
// an FP32 eigensolver, refined to FP64 accuracy by the iteration of Ogita and Aishima
// ("Iterative refinement for symmetric eigenvalue decomposition", Japan J. Indust. Appl.
// Math. 35, 2018), whose matrix products run as exact sliced GEMMs on the tensor cores.
//
// Why: FP64 arithmetic on this GPU runs at a small fraction of its bf16 tensor rate, and the
// FP64 solver (cuSOLVER Dsyevd) spends most of its time in the FP64 tridiagonalisation: 34 ms at
// n = 1000, against 11 ms for the FP32 solver.
//
// One step of the iteration, from an approximate eigenvector matrix X (columns x_i):
//   R = I - X^T X,   S = X^T Phi X,   lambda_i = S_ii / (1 - R_ii),
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   for pairs farther apart than delta,
//   E_ij = R_ij / 2                                         for closer pairs and for i = j,
//   X <- X (I + E),
// with delta = 2 (||S - diag(lambda)|| + ||Phi|| ||R||) (2-norms bounded by the maximum absolute
// row sum, ||Phi|| by max |lambda_i|), and never below 64 n u ||Phi||, the spacing below which a
// pair's vectors are not determined in FP64.  Convergence is quadratic for separated
// eigenvalues.  When the off-diagonal of S is already near the FP64 floor while R is not, the step
// uses E = R / 2 for every pair: it restores orthogonality, which for close pairs the Newton
// step's own rounding (u ||Phi|| / gap) would keep disturbing.
//
// How the products are formed.  The steps start from the FP32 solver's vectors with X^T X and
// X^T Phi X from FP64-accurate products (8 slices of 7 bits per operand, 56 bits) and X (I + E)
// formed the same way.  Once a step's correction is small (max |E| <= 1e-5), the vectors X0 of that
// step become the base: X = X0 (I + F), F the correction accumulated from then on, and
//   X^T X    = G0 + F + F^T + F^T F - R0 F - (R0 F)^T - F^T R0 F,            G0 = X0^T X0 = I - R0,
//   X^T Phi X = S0 + D0 F + (D0 F)^T + T0 F + (T0 F)^T + F^T D0 F + F^T T0 F,   S0 = X0^T Phi X0 = D0 + T0,
// D0 = diag(S0), G0 and S0 those of the base step.  The terms with F then need only the 28 bits
// of 4-slice products (their error is ~2^-28 max|F|^2 sqrt(n) < 1e-16), and F^T R0 F and
// F^T T0 F (< 1e-15 max|F|^2) are left out.  Z = X0 + X0 F is formed with an FP64-accurate
// product.  The iteration stops when max |R_ij| and max_{i != j} |S_ij| / ||Phi|| are both at most
// 16 u max(sqrt(n), 8) (u = 2^-53); Z is accepted only after the same test on Z^T Z and Z^T Phi Z
// recomputed from Z with FP64-accurate products, and the eigenvalues are S_ii / (Z^T Z)_ii of that
// recomputation.  If the test fails, the iteration has not converged after 8 steps, the FP32
// solver failed, the scratch memory is not available, or n > 2048 (where the measured steps did
// not converge), the caller computes the decomposition with the FP64 solver instead.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "gwas_internal.cuh"
#include "xgemm.cuh"

namespace {

// accurate products: 8 slices, levels 0..7, K chunks of 256 (every level sum exact); cheap
// products: 4 slices, levels 0..3, K chunks of 1024
struct RowStat {
  double sumR, sumD, maxR, maxS;  // row sums of |R| and |S - diag|, maxima of |R| and off-diagonal |S|
};

constexpr int kSlices = 8, kBits = 7, kLevels = 7, kChunk = 256, kMaxSteps = 8, kCheapSlices = 4;
// largest correction from which the steps continue incrementally
constexpr double kIncremental = 1e-5;
// Largest n refined.  Measured on kinships of 5000 markers against the FP64 solver: n = 1000
// 16.7 / 34.4 ms (4 steps), 1500 39 / 64 ms (7), 2000 73 / 101 ms (8), 2500 116 / 165 ms (6);
// at n = 3000 the steps stalled with the off-diagonal of S at twice the tolerance (the floor
// u ||Phi|| / gap of the closest pairs grows faster than sqrt(n)), and at n = 4096 and above
// they did not converge either, so those sizes go to the FP64 solver directly.
constexpr int kRefineMaxN = 2048;

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// out[j][i] = in[i][j] for an n x n matrix (32 x 32 tiles staged in shared memory).
__global__ void transpose_n_kernel(const double* __restrict__ in, int n, double* __restrict__ out) {
  __shared__ double t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y)
    if (x < n && y0 + dy < n) t[dy][threadIdx.x] = in[(size_t)(y0 + dy) * n + x];
  __syncthreads();
  const int ox = y0 + threadIdx.x, oy0 = blockIdx.x * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y)
    if (ox < n && oy0 + dy < n) out[(size_t)(oy0 + dy) * n + ox] = t[threadIdx.x][dy];
}

// Row i of R = I - G and of S - diag(lambda) (G = X^T X and S = X^T Phi X, row-major): the
// eigenvalue estimate lambda_i = S_ii / G_ii, the row's absolute sums and maxima.  A warp per row.
__global__ void refine_rows_kernel(const double* __restrict__ G, const double* __restrict__ S, int n,
                                   double* __restrict__ lam, RowStat* __restrict__ rowstat) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (i >= n) return;
  const double* g = G + (size_t)i * n;
  const double* s = S + (size_t)i * n;
  const double li = s[i] / g[i];
  double sumR = 0, sumD = 0, maxR = 0, maxS = 0;
  for (int j = lane; j < n; j += 32) {
    const double r = (i == j ? 1.0 : 0.0) - g[j];
    const double d = i == j ? s[j] - li : s[j];
    sumR += fabs(r);
    sumD += fabs(d);
    maxR = fmax(maxR, fabs(r));
    if (i != j) maxS = fmax(maxS, fabs(s[j]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sumR += __shfl_xor_sync(0xffffffffu, sumR, o);
    sumD += __shfl_xor_sync(0xffffffffu, sumD, o);
    maxR = fmax(maxR, __shfl_xor_sync(0xffffffffu, maxR, o));
    maxS = fmax(maxS, __shfl_xor_sync(0xffffffffu, maxS, o));
  }
  if (lane == 0) {
    lam[i] = li;
    rowstat[i] = RowStat{sumR, sumD, maxR, maxS};
  }
}

// out[0] = max_i sum_j |R_ij|, out[1] = max_i sum_j |(S - diag lambda)_ij|, out[2] = max |R_ij|,
// out[3] = max_{i != j} |S_ij|, out[4] = max |lambda_i|; a NaN anywhere makes out[5] nonzero.
// One block of 256 threads.
__global__ void refine_reduce_kernel(const RowStat* __restrict__ rowstat, const double* __restrict__ lam, int n,
                                     double* __restrict__ out) {
  __shared__ double sh[6][256];
  double a = 0, b = 0, c = 0, d = 0, e = 0, bad = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const RowStat v = rowstat[i];
    a = fmax(a, v.sumR);
    b = fmax(b, v.sumD);
    c = fmax(c, v.maxR);
    d = fmax(d, v.maxS);
    e = fmax(e, fabs(lam[i]));
    if (!isfinite(v.sumR) || !isfinite(v.sumD) || !isfinite(v.maxR) || !isfinite(v.maxS) || !isfinite(lam[i])) bad = 1;
  }
  sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = b; sh[2][threadIdx.x] = c;
  sh[3][threadIdx.x] = d; sh[4][threadIdx.x] = e; sh[5][threadIdx.x] = bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

// The correction E of one step, stored column-major (E[c * n + r] = E_rc) so that its columns are
// the rows the next product slices.  32 x 32 tiles: G and S read along rows, E written along
// columns.  orth != 0: E = R / 2 for every pair.
__global__ void refine_correction_kernel(const double* __restrict__ G, const double* __restrict__ S,
                                         const double* __restrict__ lam, int n, double delta, int orth,
                                         double* __restrict__ E, unsigned long long* __restrict__ emax) {
  __shared__ double t[32][33];
  __shared__ unsigned long long bmax;
  if (threadIdx.x == 0 && threadIdx.y == 0) bmax = 0;
  const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy;
    double e = 0;
    if (r < n && c < n) {
      const double rr = (r == c ? 1.0 : 0.0) - G[(size_t)r * n + c];
      const double gap = lam[c] - lam[r];
      if (r == c || orth || fabs(gap) <= delta) e = 0.5 * rr;
      else e = (S[(size_t)r * n + c] + lam[c] * rr) / gap;
    }
    t[dy][threadIdx.x] = e;
  }
  __syncthreads();
  // max |E| of the tile: |e| as an integer bit pattern orders like the value (e finite)
  unsigned long long m = 0;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(t[dy][threadIdx.x]));
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, m, o);
    m = b > m ? b : m;
  }
  if (threadIdx.x == 0) atomicMax(&bmax, m);
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) atomicMax(emax, bmax);
  const int orow = r0 + threadIdx.x, oc0 = blockIdx.x * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y)
    if (orow < n && oc0 + dy < n) E[(size_t)(oc0 + dy) * n + orow] = t[threadIdx.x][dy];
}

// Z[:, k] = X[:, perm[k]] and lam_out[k] = lam[perm[k]] (column-major n x n).
__global__ void gather_columns_kernel(const double* __restrict__ X, const double* __restrict__ lam,
                                      const int* __restrict__ perm, int n, double* __restrict__ Z,
                                      double* __restrict__ lam_out) {
  const int k = blockIdx.x;
  const int src = perm[k];
  for (int i = threadIdx.x; i < n; i += blockDim.x) Z[(size_t)k * n + i] = X[(size_t)src * n + i];
  if (threadIdx.x == 0) lam_out[k] = lam[src];
}

// From G0 = X0^T X0 and S0 = X0^T Phi X0 (row-major): R0 = I - G0, T0 = S0 - diag(S0) (row-major)
// and d = diag(S0).
__global__ void split_residuals_kernel(const double* __restrict__ G0, const double* __restrict__ S0, int n,
                                       double* __restrict__ R0, double* __restrict__ T0, double* __restrict__ d) {
  const size_t nn = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    R0[e] = (r == c ? 1.0 : 0.0) - G0[e];
    T0[e] = r == c ? 0.0 : S0[e];
    if (r == c) d[r] = S0[e];
  }
}

// DF = diag(d) F, both column-major (DF[c n + r] = d_r F_rc).
__global__ void scale_rows_kernel(const double* __restrict__ F, const double* __restrict__ d, int n,
                                  double* __restrict__ DF) {
  const size_t nn = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x)
    DF[e] = d[e % n] * F[e];
}

// X^T X and X^T Phi X of X = X0 (I + F) from the products (row-major, P[r n + c]):
//   G = G0 + F + F^T + P1 - P3 - P3^T,   S = S0 + D0 F + (D0 F)^T + P4 + P4^T + P2,
// P1 = F^T F, P2 = F^T D0 F, P3 = R0 F, P4 = T0 F; F column-major (F_rc = F[c n + r]).
__global__ void assemble_kernel(const double* __restrict__ G0, const double* __restrict__ S0,
                                const double* __restrict__ d, const double* __restrict__ F,
                                const double* __restrict__ P1, const double* __restrict__ P2,
                                const double* __restrict__ P3, const double* __restrict__ P4, int n,
                                double* __restrict__ G, double* __restrict__ S) {
  const size_t nn = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    const size_t t = (size_t)c * n + r;  // the transposed position
    const double frc = F[t], fcr = F[e];
    G[e] = G0[e] + (frc + fcr) + P1[e] - (P3[e] + P3[t]);
    S[e] = S0[e] + (d[r] * frc + d[c] * fcr) + (P4[e] + P4[t]) + P2[e];
  }
}

// F = a F + E (column-major, elementwise; a = 0 on the first step).
__global__ void axpy_kernel(double a, double* __restrict__ F, const double* __restrict__ E, size_t N) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
    F[e] = (a == 0.0 ? 0.0 : a * F[e]) + E[e];
}

int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace


int eig_refined(gwas_ctx* c, void* solver, const double* phi, int n, double* Z, double* lam, int* steps) {
  cusolverDnHandle_t h = (cusolverDnHandle_t)solver;
  constexpr int kFallBack = EIG_FALL_BACK;
  *steps = 0;
  if (n > kRefineMaxN) return kFallBack;
  const size_t nn = (size_t)n * n;
  const int Np = (int)rup(n, 128), Kpad = (int)rup(n, 64);
  const size_t planes8 = (size_t)kSlices * Np * Kpad, planes4 = (size_t)kCheapSlices * Np * Kpad;
  std::vector<void*> bufs;
  // scratch that does not fit (an HBM budget, a full device) leaves the FP64 solver to do the work
  auto alloc = [&](size_t bytes, void** p) {
    const int rc = ctx_alloc(c, bytes, p);
    if (rc == GWAS_OK) bufs.push_back(*p);
    return rc == GWAS_OK ? GWAS_OK : kFallBack;
  };
  auto done = [&](int rc) {
    cudaStreamSynchronize(c->stream);
    for (void* p : bufs) ctx_free(c, p);
    return rc;
  };
  float *A32 = nullptr, *w32 = nullptr, *work = nullptr;
  int *info = nullptr, *perm = nullptr;
  double *X = nullptr, *G0 = nullptr, *S0 = nullptr, *G = nullptr, *S = nullptr, *F = nullptr, *E = nullptr;
  double *W[4] = {nullptr, nullptr, nullptr, nullptr}, *d = nullptr, *lt = nullptr, *stats = nullptr;
  double *sphi = nullptr, *sa = nullptr, *sb = nullptr, *sR = nullptr, *sT = nullptr, *sF = nullptr, *sD = nullptr;
  RowStat* rowstat = nullptr;
  __nv_bfloat16 *Pphi = nullptr, *PA = nullptr, *PB = nullptr, *PR = nullptr, *PT = nullptr, *PF = nullptr,
                *PD = nullptr;
  int rc, lwork = 0;
  if ((rc = alloc(sizeof(float) * nn, (void**)&A32)) || (rc = alloc(sizeof(float) * n, (void**)&w32)))
    return done(rc);
  if (cusolverDnSsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A32, n, w32, &lwork) !=
      CUSOLVER_STATUS_SUCCESS)
    return done(kFallBack);
  if ((rc = alloc(sizeof(float) * std::max(lwork, 1), (void**)&work)) || (rc = alloc(sizeof(int), (void**)&info)) ||
      (rc = alloc(sizeof(int) * n, (void**)&perm)))
    return done(rc);
  for (double** b : {&X, &G0, &S0, &G, &S, &F, &E, &W[0], &W[1], &W[2], &W[3]})
    if ((rc = alloc(sizeof(double) * nn, (void**)b))) return done(rc);
  for (double** b : {&d, &lt})
    if ((rc = alloc(sizeof(double) * n, (void**)b))) return done(rc);
  for (double** b : {&sphi, &sa, &sb, &sR, &sT, &sF, &sD})
    if ((rc = alloc(sizeof(double) * Np, (void**)b))) return done(rc);
  if ((rc = alloc(sizeof(double) * 8, (void**)&stats)) || (rc = alloc(sizeof(RowStat) * n, (void**)&rowstat)))
    return done(rc);
  for (__nv_bfloat16** b : {&Pphi, &PA, &PB})
    if ((rc = alloc(sizeof(__nv_bfloat16) * planes8, (void**)b))) return done(rc);
  for (__nv_bfloat16** b : {&PR, &PT, &PF, &PD})
    if ((rc = alloc(sizeof(__nv_bfloat16) * planes4, (void**)b))) return done(rc);

  const unsigned eb = (unsigned)std::min<size_t>((nn + 255) / 256, 4096);
  {
    ProfScope ps(c, "eig_fp32_solver");
    f64_to_f32_kernel<<<eb, 256, 0, c->stream>>>(phi, A32, nn);
    c->launches++;
    if (cusolverDnSsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A32, n, w32, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS)
      return done(kFallBack);
    f32_to_f64_kernel<<<eb, 256, 0, c->stream>>>(A32, X, nn);
    c->launches++;
  }

  // out (row-major n x n, out[r n + c]) = sum_k A_r[k] B_c[k] over the rows of the two sliced
  // operands; add != 0 adds to out
  auto gemm = [&](int slices, const __nv_bfloat16* A, const double* sA, const __nv_bfloat16* B, const double* sB,
                  double* out, int add) {
    XgemmArgs g{};
    g.rows = n;
    g.cols = n;
    g.rowsA_pad = Np;
    g.rowsB_pad = Np;
    g.Kpad = Kpad;
    g.level_scale = std::ldexp(1.0, -kBits);
    g.scaleA = sA;
    g.scaleB = sB;
    g.out64 = out;
    g.ldo = n;
    g.status = c->d_status;
    g.untimed = 1;
    g.kchunk = slices == kSlices ? kChunk : 0;
    g.add_to_out = add;
    return slices == kSlices ? launch_xgemm(c, kSlices, kSlices, kLevels, g, A, B)
                             : launch_xgemm(c, kCheapSlices, kCheapSlices, 3, g, A, B);
  };
  // rows of a row-major (or the columns of a column-major) n x n matrix into slice planes
  auto slice = [&](const double* M, int slices, __nv_bfloat16* P, double* sc) {
    launch_slice_rows(c, M, n, n, n, Np, Kpad, slices, kBits, P, sc, nullptr);
  };
  // G = X^T X and S = X^T Phi X of the vectors X (column-major), FP64-accurate
  auto residuals = [&](const double* Xv, double* Gout, double* Sout) {
    slice(Xv, kSlices, PA, sa);                                        // columns of X
    if ((rc = gemm(kSlices, PA, sa, PA, sa, Gout, 0))) return rc;      // X^T X
    if ((rc = gemm(kSlices, PA, sa, Pphi, sphi, W[0], 0))) return rc;  // Q = X^T Phi
    slice(W[0], kSlices, PB, sb);                                      // rows of Q
    return gemm(kSlices, PB, sb, PA, sa, Sout, 0);                     // Q X
  };
  // the statistics of (G, S) on the host: {max row sum |R|, max row sum |S - diag|, max |R|,
  // max off-diagonal |S|, max |lambda|, any non-finite}; lambda_i = S_ii / G_ii into lt
  double hs[6];
  auto statistics = [&](const double* Gv, const double* Sv) {
    refine_rows_kernel<<<(n + 7) / 8, 256, 0, c->stream>>>(Gv, Sv, n, lt, rowstat);
    refine_reduce_kernel<<<1, 256, 0, c->stream>>>(rowstat, lt, n, stats);
    c->launches += 2;
    int hinfo = 0;
    unsigned long long hstatus = 0;
    if (!ctx_cuda_ok(c, cudaMemcpyAsync(hs, stats, sizeof hs, cudaMemcpyDeviceToHost, c->stream), "refine", &rc) ||
        !ctx_cuda_ok(c, cudaMemcpyAsync(&hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, c->stream), "refine",
                     &rc) ||
        !ctx_cuda_ok(c, cudaMemcpyAsync(&hstatus, c->d_status, sizeof hstatus, cudaMemcpyDeviceToHost, c->stream),
                     "refine", &rc) ||
        !ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "refine", &rc))
      return rc;
    if (hstatus) return ctx_fail(c, GWAS_ERR_TIMEOUT, "eigendecomposition: a bounded wait expired");
    if (hinfo != 0 || hs[5] != 0) return kFallBack;  // the FP32 solver failed, or non-finite values
    return GWAS_OK;
  };
  const char* tr = std::getenv("GWAS_EIG_TRACE");
  const bool trace = tr && std::strcmp(tr, "1") == 0;
  const double u = std::ldexp(1.0, -53), tol = 16 * u * std::max(std::sqrt((double)n), 8.0);
  auto converged = [&]() { return hs[2] <= tol && hs[3] <= tol * hs[4]; };
  const dim3 tb(32, 8), tg((n + 31) / 32, (n + 31) / 32);

  slice(phi, kSlices, Pphi, sphi);  // Phi is symmetric: its columns are its rows
  unsigned long long* emax = reinterpret_cast<unsigned long long*>(stats + 6);
  bool incremental = false;
  for (int step = 0;; ++step) {
    const double* Gv = G0;
    const double* Sv = S0;
    {
      ProfScope ps(c, "eig_refine_residuals");
      if (!incremental) {
        // X^T X and X^T Phi X of the current vectors, FP64-accurate
        if ((rc = residuals(X, G0, S0))) return done(rc);
      } else {
        // those of X0 (I + F) from 4-slice products of F
        scale_rows_kernel<<<eb, 256, 0, c->stream>>>(F, d, n, E);  // E <- D0 F (scratch)
        c->launches++;
        slice(F, kCheapSlices, PF, sF);  // columns of F
        slice(E, kCheapSlices, PD, sD);  // columns of D0 F
        if ((rc = gemm(kCheapSlices, PF, sF, PF, sF, W[0], 0)) ||  // P1 = F^T F
            (rc = gemm(kCheapSlices, PF, sF, PD, sD, W[1], 0)) ||  // P2 = F^T D0 F
            (rc = gemm(kCheapSlices, PR, sR, PF, sF, W[2], 0)) ||  // P3 = R0 F
            (rc = gemm(kCheapSlices, PT, sT, PF, sF, W[3], 0)))    // P4 = T0 F
          return done(rc);
        assemble_kernel<<<eb, 256, 0, c->stream>>>(G0, S0, d, F, W[0], W[1], W[2], W[3], n, G, S);
        c->launches++;
        Gv = G;
        Sv = S;
      }
    }
    if ((rc = statistics(Gv, Sv))) return done(rc);
    *steps = step;
    if (trace)
      std::fprintf(stderr, "eig step %d%s: max|R| %.3e max|S offdiag| %.3e row sums %.3e %.3e max|lambda| %.6e\n",
                   step, incremental ? " (incremental)" : "", hs[2], hs[3], hs[0], hs[1], hs[4]);
    if (converged()) break;
    if (step == kMaxSteps) return done(kFallBack);
    const int orth = (hs[3] <= 100 * tol * hs[4] && hs[2] > tol) ? 1 : 0;
    const double delta = std::max(2 * (hs[1] + hs[4] * hs[0]), 64.0 * n * u * hs[4]);
    ProfScope ps(c, "eig_refine_update");
    unsigned long long hmax = 0;
    cudaMemsetAsync(emax, 0, sizeof *emax, c->stream);
    refine_correction_kernel<<<tg, tb, 0, c->stream>>>(Gv, Sv, lt, n, delta, orth, E, emax);
    c->launches++;
    if (!incremental) {
      if (!ctx_cuda_ok(c, cudaMemcpyAsync(&hmax, emax, sizeof hmax, cudaMemcpyDeviceToHost, c->stream), "refine",
                       &rc) ||
          !ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "refine", &rc))
        return done(rc);
    }
    const double max_e = __builtin_bit_cast(double, hmax);
    if (!incremental && max_e <= kIncremental) {
      // the current vectors become the base X0 of the incremental steps: F = E
      split_residuals_kernel<<<eb, 256, 0, c->stream>>>(G0, S0, n, W[1], W[2], d);
      c->launches++;
      slice(W[1], kCheapSlices, PR, sR);
      slice(W[2], kCheapSlices, PT, sT);
      cudaMemcpyAsync(F, E, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->stream);
      incremental = true;
    } else if (!incremental) {
      // X <- X + X E, FP64-accurate: out[r][c] = sum_k E_kr X_ck = (X E)_cr lands at X's
      // column-major position of (c, r)
      transpose_n_kernel<<<tg, tb, 0, c->stream>>>(X, n, W[0]);  // rows of X
      c->launches++;
      slice(W[0], kSlices, PB, sb);
      slice(E, kSlices, PA, sa);  // columns of E
      if ((rc = gemm(kSlices, PA, sa, PB, sb, X, 1))) return done(rc);
    } else {
      // F <- F + E + F E from the slices of the old F (the same placement as above)
      transpose_n_kernel<<<tg, tb, 0, c->stream>>>(F, n, W[0]);  // rows of F
      c->launches++;
      slice(W[0], kCheapSlices, PF, sF);
      slice(E, kCheapSlices, PD, sD);  // columns of E
      axpy_kernel<<<eb, 256, 0, c->stream>>>(1.0, F, E, nn);
      c->launches++;
      if ((rc = gemm(kCheapSlices, PD, sD, PF, sF, F, 1))) return done(rc);
    }
  }
  if (incremental) {
    {
      ProfScope ps(c, "eig_refine_update");
      // Z = X0 + X0 F, FP64-accurate
      transpose_n_kernel<<<tg, tb, 0, c->stream>>>(X, n, W[0]);  // rows of X0
      c->launches++;
      slice(W[0], kSlices, PB, sb);
      slice(F, kSlices, PA, sa);  // columns of F
      if ((rc = gemm(kSlices, PA, sa, PB, sb, X, 1))) return done(rc);
    }
    // Z is accepted on its own FP64-accurate residuals, which also give the eigenvalues
    ProfScope ps(c, "eig_refine_residuals");
    if ((rc = residuals(X, G, S))) return done(rc);
    if ((rc = statistics(G, S))) return done(rc);
    if (trace) std::fprintf(stderr, "eig check of Z: max|R| %.3e max|S offdiag| %.3e\n", hs[2], hs[3]);
    if (!converged()) return done(kFallBack);
  }
  // ascending eigenvalues, as the FP64 solver returns them
  std::vector<double> hl(n);
  if (!ctx_cuda_ok(c, cudaMemcpyAsync(hl.data(), lt, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "refine",
                   &rc) ||
      !ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "refine", &rc))
    return done(rc);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hl[a] < hl[b]; });
  if (!ctx_cuda_ok(c, cudaMemcpyAsync(perm, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream),
                   "refine", &rc))
    return done(rc);
  gather_columns_kernel<<<n, 256, 0, c->stream>>>(X, lt, perm, n, Z, lam);
  c->launches++;
  return done(GWAS_OK);
}
