// Plain FP64 path of Algorithm 5 (Section 3): the rotations by Z^T, the per-trait
// operations and the per-pair contractions + p x p SPD solve, all in FP64 on the
// CUDA cores.  This is the paper's own arithmetic (Section 6 runs in double
// precision) and the reference point of the mixed-precision path.
#include <cstdint>

#include "gwas_internal.cuh"

namespace {

// ------------------------------------------------------------------ rotation GEMM
// C[r][col] = sum_k A[r][k] * Z[k][col]; Z is n x n column-major, so the column col of
// Z (eigenvector col) is contiguous: Z[k][col] = Zc[col * n + k].
constexpr int RT = 64, RK = 16;

template <typename TA>
__global__ void __launch_bounds__(256) rotate_fp64_kernel(const TA* __restrict__ A, int64_t rows, int64_t lda,
                                                          const double* __restrict__ Zc, int n, double* __restrict__ C) {
  __shared__ double As[RK][RT + 1];
  __shared__ double Bs[RK][RT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t r0 = (int64_t)blockIdx.x * RT;
  const int c0 = blockIdx.y * RT;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += RK) {
    for (int e = threadIdx.x; e < RT * RK; e += 256) {
      int rr = e / RK, kk = e % RK;
      int64_t r = r0 + rr;
      int k = k0 + kk;
      As[kk][rr] = (r < rows && k < n) ? (double)A[r * lda + k] : 0.0;
      int cc = e / RK;
      int col = c0 + cc;
      Bs[kk][cc] = (col < n && k < n) ? Zc[(size_t)col * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = Bs[kk][tx + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t r = r0 + ty + 16 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int col = c0 + tx + 16 * j;
      if (col < n) C[r * n + col] = acc[i][j];
    }
  }
}

// The same product for a few rows (the covariates X_L, at setup): one warp per output C[r][col], a dot
// product of row r of A with eigenvector col (contiguous in Zc).  The 64-row tiles of the
// kernel above would spend 64/rows times the FP64 work of this product.
template <typename TA>
__global__ void __launch_bounds__(256) rotate_rows_kernel(const TA* __restrict__ A, int64_t rows, int64_t lda,
                                                          const double* __restrict__ Zc, int n, double* __restrict__ C) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (w >= rows * n) return;
  const int64_t r = w / n;
  const int col = (int)(w % n);
  const double* z = Zc + (size_t)col * n;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc = fma((double)A[r * lda + k], z[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) C[r * n + col] = acc;
}

template <typename TA>
void rotate(gwas_ctx* c, const TA* A, int64_t rows, int64_t lda, double* C) {
  if (rows <= 0) return;
  dim3 grid((unsigned)((rows + RT - 1) / RT), (c->n + RT - 1) / RT);
  ProfScope ps(c, "rotate_fp64");
  rotate_fp64_kernel<TA><<<grid, 256, 0, c->stream>>>(A, rows, lda, c->Z, c->n, C);
  c->launches++;
}

// ------------------------------------------------------------------ per-trait prep
// Algorithm 5 per-trait lines with the weight e_j = diag(D_j^-1) (K_j K_j^T = D_j^-1,
// D_j = h_j^2 Lambda + (1 - h_j^2) I; sigma_j^2 omitted, b does not depend on it):
//   R[j] = [e∘y'_j | e∘x'_L,1 .. e∘x'_L,p-1 | e]            ([t][p+1][n])
// and the per-trait part of the Cholesky factorisation of every pair's p x p matrix
// S = [[S_TL, S_BL^T], [S_BL, S_BR]] (Algorithm 5's posv; its leading block S_TL does not
// depend on the SNP, so it is factored once per trait):
//   consts[j] = {L (p-1 x p-1, row-major, zero above the diagonal): L L^T = S_TL = X'_L^T diag(e) X'_L,
//                g = L^-1 b_T with b_T = X'_L^T (e∘y'),  rr = y'^T diag(e) y' - g^T g}
__global__ void __launch_bounds__(256) prep_fp64_kernel(const double* __restrict__ Yt, const double* __restrict__ h2,
                                                        const double* __restrict__ lam, const double* __restrict__ XLt,
                                                        int n, int pm1, double* __restrict__ R,
                                                        double* __restrict__ consts, int cst) {
  const int j = blockIdx.x;
  const int p = pm1 + 1;
  const double h = h2[j];
  const double* y = Yt + (size_t)j * n;
  double* Rj = R + (size_t)j * (p + 1) * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double e = 1.0 / (h * lam[k] + (1.0 - h));
    Rj[k] = e * y[k];
    Rj[(size_t)p * n + k] = e;
    for (int a = 0; a < pm1; ++a) Rj[(size_t)(1 + a) * n + k] = e * XLt[(size_t)a * n + k];
  }
  __syncthreads();  // the block's global writes of R are visible to all its threads
  // the lower triangle of S_TL, then b_T, then y'^T diag(e) y': one inner product over k per
  // entry, a warp per entry
  __shared__ double sh[GWAS_MAX_PM1 * (GWAS_MAX_PM1 + 1) / 2 + GWAS_MAX_PM1 + 1];
  const int ntri = pm1 * (pm1 + 1) / 2, ns = ntri + pm1 + 1;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int q = warp; q < ns; q += blockDim.x / 32) {
    const double *u, *v;
    if (q < ntri) {
      int a = 0;
      while ((a + 1) * (a + 2) / 2 <= q) ++a;
      const int b = q - a * (a + 1) / 2;
      u = Rj + (size_t)(1 + a) * n;
      v = XLt + (size_t)b * n;
    } else if (q < ntri + pm1) {
      u = Rj + (size_t)(1 + q - ntri) * n;
      v = y;
    } else {
      u = Rj;
      v = y;
    }
    double acc = 0.0;
    for (int k = lane; k < n; k += 32) acc = fma(u[k], v[k], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* L = consts + (size_t)j * cst;
    double* g = L + pm1 * pm1;
    for (int a = 0; a < pm1; ++a) {
      for (int b = 0; b <= a; ++b) {
        double v = sh[a * (a + 1) / 2 + b];
        for (int k = 0; k < b; ++k) v -= L[a * pm1 + k] * L[b * pm1 + k];
        L[a * pm1 + b] = a == b ? sqrt(v > 0 ? v : 1e-300) : v / L[b * pm1 + b];
      }
      for (int b = a + 1; b < pm1; ++b) L[a * pm1 + b] = 0.0;
    }
    double gg = 0.0;
    for (int a = 0; a < pm1; ++a) {
      double v = sh[ntri + a];
      for (int k = 0; k < a; ++k) v -= L[a * pm1 + k] * g[k];
      g[a] = v / L[a * pm1 + a];
      gg += g[a] * g[a];
    }
    g[pm1] = sh[ns - 1] - gg;
  }
}

// ------------------------------------------------------------------ fused contraction + solve
// For each pair (i, j): with W_R = K_j x'_i (Algorithm 5, never formed: K_j K_j^T = diag(e)),
//   b_B  = x'_i^T (e∘y'_j)   S_BL = x'_i^T (e∘X'_L)   S_BR = x'_i^T diag(e) x'_i
// then the last row of the Cholesky factor of S (the Schur complement of S_TL, Algorithm 2's
// blocks): z = L^-1 S_BL, delta = S_BR - z^T z; the solve b = S^-1 c with c = [b_T; b_B]:
//   beta = (b_B - z^T g) / delta,   b_L = L^-T (g - z beta),   RSS = rr - (b_B - z^T g) beta.
// Block tile: FT_S SNPs x FT_T traits, each thread MA SNPs x MB traits with p + 1 FP64
// accumulators per pair (64 x 16 and 2 x 2 up to p = 8, 32 x 8 and 1 x 1 above); the k extent of a stage shrinks as p grows to keep the shared tiles
// under 48 KB.
__host__ __device__ constexpr int fp64_ma(int pm1) { return pm1 <= 7 ? 2 : 1; }   // SNPs per thread
__host__ __device__ constexpr int fp64_fs(int pm1) { return 32 * fp64_ma(pm1); }  // SNPs per block
__host__ __device__ constexpr int fp64_mb(int pm1) { return pm1 <= 7 ? 2 : 1; }   // traits per thread
__host__ __device__ constexpr int fp64_ft(int pm1) { return 8 * fp64_mb(pm1); }   // traits per block
__host__ __device__ constexpr int fp64_fk(int pm1) { return pm1 <= 3 ? 32 : 16; } // k per stage

template <int PM1>
__global__ void __launch_bounds__(256) fused_fp64_kernel(const double* __restrict__ Xt, int n, int64_t i0, int64_t i1,
                                                         int tb, const double* __restrict__ R,
                                                         const double* __restrict__ consts, int cst, int full_b,
                                                         int64_t ldo, void* out_b, float* out_se,
                                                         unsigned long long* singular) {
  constexpr int P = PM1 + 1, Q1 = PM1 > 0 ? PM1 : 1;
  constexpr int NV = P + 1;  // accumulated values per pair
  constexpr int MA = fp64_ma(PM1), FT_S = fp64_fs(PM1), MB = fp64_mb(PM1), FT_T = fp64_ft(PM1), FK = fp64_fk(PM1);
  static_assert((FK * (FT_S + 1) + FK * (FT_T * NV + 1)) * 8 <= 48 * 1024, "static shared memory");
  __shared__ double xs[FK][FT_S + 1];
  __shared__ double rs[FK][FT_T * NV + 1];
  const int tx = threadIdx.x % 8;    // trait group: traits tx + 8 b
  const int ty = threadIdx.x / 8;    // SNP group:   SNPs ty + 32 a
  const int64_t s0 = i0 + (int64_t)blockIdx.x * FT_S;
  const int jt0 = blockIdx.y * FT_T;
  double acc[MA][MB][NV];
#pragma unroll
  for (int a = 0; a < MA; ++a)
#pragma unroll
    for (int b = 0; b < MB; ++b)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[a][b][v] = 0.0;
  for (int k0 = 0; k0 < n; k0 += FK) {
    for (int e = threadIdx.x; e < FT_S * FK; e += 256) {
      int ss = e / FK, kk = e % FK;
      int64_t s = s0 + ss;
      int k = k0 + kk;
      xs[kk][ss] = (s < i1 && k < n) ? Xt[s * n + k] : 0.0;
    }
    for (int e = threadIdx.x; e < FT_T * NV * FK; e += 256) {
      int row = e / FK, kk = e % FK;
      int jj = row / NV, v = row % NV;
      int j = jt0 + jj, k = k0 + kk;
      rs[kk][jj * NV + v] = (j < tb && k < n) ? R[((size_t)j * NV + v) * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < FK; ++kk) {
      double x[MA];
#pragma unroll
      for (int a = 0; a < MA; ++a) x[a] = xs[kk][ty + 32 * a];
#pragma unroll
      for (int b = 0; b < MB; ++b) {
        const double* r = &rs[kk][(tx + 8 * b) * NV];
#pragma unroll
        for (int a = 0; a < MA; ++a) {
#pragma unroll
          for (int v = 0; v < P; ++v) acc[a][b][v] = fma(x[a], r[v], acc[a][b][v]);
          acc[a][b][P] = fma(x[a] * x[a], r[P], acc[a][b][P]);
        }
      }
    }
    __syncthreads();
  }
  const int p = P;
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int jj = jt0 + tx + 8 * b;
    if (jj >= tb) continue;
    const double* L = consts + (size_t)jj * cst;  // L (row-major), g, rr
    const double* g = L + PM1 * PM1;
#pragma unroll
    for (int a = 0; a < MA; ++a) {
      const int64_t s = s0 + ty + 32 * a;
      if (s >= i1) continue;
      // last row of the Cholesky factor of S: z = L^-1 S_BL, l_pp^2 = delta = S_BR - z^T z
      double z[Q1];
      double zz = 0.0, zg = 0.0;
#pragma unroll
      for (int c = 0; c < PM1; ++c) {
        double v = acc[a][b][1 + c];
#pragma unroll
        for (int d = 0; d < c; ++d) v -= L[c * PM1 + d] * z[d];
        z[c] = v / L[c * PM1 + c];
        zz = fma(z[c], z[c], zz);
        zg = fma(z[c], g[c], zg);
      }
      const double sbr = acc[a][b][P];
      const double delta = sbr - zz;
      const bool ok = delta > 1e-10 * sbr;
      const double lpp = sqrt(delta > 0 ? delta : 1e-300);
      // forward and back substitution with [[L, 0], [z^T, l_pp]]
      const double num = acc[a][b][0] - zg;
      const double beta = num / (lpp * lpp);
      const double rss = g[PM1] - num * beta;
      double se = sqrt(fmax(rss, 0.0) / (double)(n - p)) / lpp;
      double bb[P];
      bb[PM1] = beta;
      if (full_b) {
#pragma unroll
        for (int c = PM1 - 1; c >= 0; --c) {
          double v = g[c] - z[c] * beta;
#pragma unroll
          for (int w = c + 1; w < PM1; ++w) v -= L[w * PM1 + c] * bb[w];
          bb[c] = v / L[c * PM1 + c];
        }
      }
      if (!ok) {
        atomicAdd(singular, 1ull);
#pragma unroll
        for (int u = 0; u < P; ++u) bb[u] = __longlong_as_double(0x7ff8000000000000ll);
        se = bb[0];
      }
      const int64_t o = (int64_t)jj * ldo + (s - i0);
      if (full_b) {
        double* ob = (double*)out_b + o * P;
#pragma unroll
        for (int u = 0; u < P; ++u) ob[u] = bb[u];
      } else {
        ((float*)out_b)[o] = (float)bb[PM1];
        out_se[o] = (float)se;
      }
    }
  }
}

}  // namespace

int consts_stride(int pm1) { return pm1 * pm1 + pm1 + 1; }

void launch_rotate_fp64_i8(gwas_ctx* c, const int8_t* A, int64_t rows, int64_t lda, double* C) {
  rotate<int8_t>(c, A, rows, lda, C);
}
void launch_rotate_fp64_f64(gwas_ctx* c, const double* A, int64_t rows, int64_t lda, double* C) {
  rotate<double>(c, A, rows, lda, C);
}
void launch_rotate_fp64_rows(gwas_ctx* c, const double* A, int64_t rows, int64_t lda, double* C) {
  if (rows <= 0) return;
  const int64_t warps = rows * (int64_t)c->n;
  ProfScope ps(c, "rotate_fp64");
  rotate_rows_kernel<double><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c->stream>>>(A, rows, lda, c->Z, c->n, C);
  c->launches++;
}

void launch_prep_fp64(gwas_ctx* c, const double* Yt, int tb, const double* h2, double* R, double* consts) {
  ProfScope ps(c, "prep_fp64");
  prep_fp64_kernel<<<tb, 256, 0, c->stream>>>(Yt, h2, c->lam, c->XLt, c->n, c->pm1, R, consts, consts_stride(c->pm1));
  c->launches++;
}

void launch_fused_fp64(gwas_ctx* c, int64_t i0, int64_t i1, int j0, int tb, int64_t ldo, const double* R,
                       const double* consts, void* out) {
  (void)j0;
  void* ob = out;
  float* os = nullptr;
  int full = c->output == GWAS_OUT_FULL_B;
  if (!full) {
    void** pr = (void**)out;
    ob = pr[0];
    os = (float*)pr[1];
  }
  const int ft = fp64_ft(c->pm1), fs = fp64_fs(c->pm1);
  dim3 grid((unsigned)((i1 - i0 + fs - 1) / fs), (tb + ft - 1) / ft);
  unsigned long long* sing = c->d_status + 1;
  const int cst = consts_stride(c->pm1);
  ProfScope ps(c, "fused_fp64");
#define GWAS_FUSED_CASE(K)                                                                                      \
  case K:                                                                                                       \
    fused_fp64_kernel<K><<<grid, 256, 0, c->stream>>>(c->Xt, c->n, i0, i1, tb, R, consts, cst, full, ldo, ob, os, \
                                                      sing);                                                    \
    break;
  switch (c->pm1) {
    GWAS_FUSED_CASE(0) GWAS_FUSED_CASE(1) GWAS_FUSED_CASE(2) GWAS_FUSED_CASE(3) GWAS_FUSED_CASE(4)
    GWAS_FUSED_CASE(5) GWAS_FUSED_CASE(6) GWAS_FUSED_CASE(7) GWAS_FUSED_CASE(8) GWAS_FUSED_CASE(9)
    GWAS_FUSED_CASE(10) GWAS_FUSED_CASE(11) GWAS_FUSED_CASE(12) GWAS_FUSED_CASE(13) GWAS_FUSED_CASE(14)
    GWAS_FUSED_CASE(15) GWAS_FUSED_CASE(16) GWAS_FUSED_CASE(17) GWAS_FUSED_CASE(18) GWAS_FUSED_CASE(19)
  }
#undef GWAS_FUSED_CASE
  c->launches++;
}
