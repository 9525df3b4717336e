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
//   consts[j] = {S_TL = X'_L^T diag(e) X'_L (row-major), b_T = X'_L^T (e∘y'_j), yy = y'^T diag(e) y'}
__global__ void __launch_bounds__(256) prep_fp64_kernel(const double* __restrict__ Yt, const double* __restrict__ h2,
                                                        const double* __restrict__ lam, const double* __restrict__ XLt,
                                                        int n, int pm1, double* __restrict__ R,
                                                        double* __restrict__ consts, int cst) {
  const int j = blockIdx.x;
  const int p = pm1 + 1;
  const double h = h2[j];
  const double* y = Yt + (size_t)j * n;
  double* Rj = R + (size_t)j * (p + 1) * n;
  // partial sums: S_TL (pm1*pm1), b_T (pm1), yy (1)
  double part[GWAS_MAX_PM1 * GWAS_MAX_PM1 + GWAS_MAX_PM1 + 1];
  const int ns = pm1 * pm1 + pm1 + 1;
  for (int q = 0; q < ns; ++q) part[q] = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double e = 1.0 / (h * lam[k] + (1.0 - h));
    double yk = y[k];
    Rj[k] = e * yk;
    Rj[(size_t)p * n + k] = e;
    double xl[GWAS_MAX_PM1];
    for (int a = 0; a < pm1; ++a) {
      xl[a] = XLt[(size_t)a * n + k];
      Rj[(size_t)(1 + a) * n + k] = e * xl[a];
    }
    for (int a = 0; a < pm1; ++a) {
      for (int b = 0; b < pm1; ++b) part[a * pm1 + b] += e * xl[a] * xl[b];
      part[pm1 * pm1 + a] += e * xl[a] * yk;
    }
    part[ns - 1] += e * yk * yk;
  }
  __shared__ double red[8][GWAS_MAX_PM1 * GWAS_MAX_PM1 + GWAS_MAX_PM1 + 1];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int q = 0; q < ns; ++q) {
    double v = part[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < ns) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w][threadIdx.x];
    consts[(size_t)j * cst + threadIdx.x] = v;
  }
}

// ------------------------------------------------------------------ fused contraction + solve
// For each pair (i, j): with W_R = K_j x'_i (Algorithm 5, never formed: K_j K_j^T = diag(e)),
//   b_B  = x'_i^T (e∘y'_j)   S_BL = x'_i^T (e∘X'_L)   S_BR = x'_i^T diag(e) x'_i
// then S = [[S_TL, S_BL^T], [S_BL, S_BR]], c = [b_T; b_B] and b = S^-1 c by Cholesky (posv).
constexpr int FT_S = 64;   // SNPs per block
constexpr int FT_T = 16;   // traits per block
constexpr int FK = 32;     // k per stage

template <int PM1>
__global__ void __launch_bounds__(256) fused_fp64_kernel(const double* __restrict__ Xt, int n, int64_t i0, int64_t i1,
                                                         int tb, const double* __restrict__ R,
                                                         const double* __restrict__ consts, int cst, int full_b,
                                                         int64_t ldo, void* out_b, float* out_se,
                                                         unsigned long long* singular) {
  constexpr int P = PM1 + 1;
  constexpr int NV = P + 1;  // accumulated values per pair
  __shared__ double xs[FK][FT_S + 1];
  __shared__ double rs[FK][FT_T * NV + 1];
  const int tx = threadIdx.x % 8;    // trait group: traits tx, tx+8
  const int ty = threadIdx.x / 8;    // SNP group:   SNPs ty, ty+32
  const int64_t s0 = i0 + (int64_t)blockIdx.x * FT_S;
  const int jt0 = blockIdx.y * FT_T;
  double acc[2][2][NV];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
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
      double x[2] = {xs[kk][ty], xs[kk][ty + 32]};
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const double* r = &rs[kk][(tx + 8 * b) * NV];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
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
  for (int b = 0; b < 2; ++b) {
    const int jj = jt0 + tx + 8 * b;
    if (jj >= tb) continue;
    const double* cj = consts + (size_t)jj * cst;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int64_t s = s0 + ty + 32 * a;
      if (s >= i1) continue;
      // assemble S (lower triangle) and c
      double S[P][P], c[P];
#pragma unroll
      for (int u = 0; u < PM1; ++u) {
#pragma unroll
        for (int w = 0; w < PM1; ++w) S[u][w] = cj[u * PM1 + w];
        S[PM1][u] = acc[a][b][1 + u];
        S[u][PM1] = acc[a][b][1 + u];
        c[u] = cj[PM1 * PM1 + u];
      }
      S[PM1][PM1] = acc[a][b][P];
      c[PM1] = acc[a][b][0];
      const double yy = cj[PM1 * PM1 + PM1];
      // Cholesky S = L L^T in place (lower)
      bool ok = true;
#pragma unroll
      for (int u = 0; u < P; ++u) {
        double d = S[u][u];
#pragma unroll
        for (int w = 0; w < u; ++w) d -= S[u][w] * S[u][w];
        if (u == PM1) ok = d > 1e-10 * S[u][u];
        double l = sqrt(d > 0 ? d : 1e-300);
        S[u][u] = l;
#pragma unroll
        for (int r = u + 1; r < P; ++r) {
          double v = S[r][u];
#pragma unroll
          for (int w = 0; w < u; ++w) v -= S[r][w] * S[u][w];
          S[r][u] = v / l;
        }
      }
      double z[P], bb[P];
#pragma unroll
      for (int u = 0; u < P; ++u) {
        double v = c[u];
#pragma unroll
        for (int w = 0; w < u; ++w) v -= S[u][w] * z[w];
        z[u] = v / S[u][u];
      }
#pragma unroll
      for (int u = P - 1; u >= 0; --u) {
        double v = z[u];
#pragma unroll
        for (int w = u + 1; w < P; ++w) v -= S[w][u] * bb[w];
        bb[u] = v / S[u][u];
      }
      // RSS = v^T v - c^T b, [S^-1]_pp = 1 / L_pp^2
      double ctb = 0;
#pragma unroll
      for (int u = 0; u < P; ++u) ctb += c[u] * bb[u];
      double rss = yy - ctb;
      double lpp = S[PM1][PM1];
      double se = sqrt(fmax(rss, 0.0) / (double)(n - p)) / lpp;
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
  dim3 grid((unsigned)((i1 - i0 + FT_S - 1) / FT_S), (tb + FT_T - 1) / FT_T);
  unsigned long long* sing = c->d_status + 1;
  const int cst = consts_stride(c->pm1);
  ProfScope ps(c, "fused_fp64");
#define GWAS_FUSED_CASE(K)                                                                                      \
  case K:                                                                                                       \
    fused_fp64_kernel<K><<<grid, 256, 0, c->stream>>>(c->Xt, c->n, i0, i1, tb, R, consts, cst, full, ldo, ob, os, \
                                                      sing);                                                    \
    break;
  switch (c->pm1) {
    GWAS_FUSED_CASE(0) GWAS_FUSED_CASE(1) GWAS_FUSED_CASE(2) GWAS_FUSED_CASE(3)
    GWAS_FUSED_CASE(4) GWAS_FUSED_CASE(5) GWAS_FUSED_CASE(6) GWAS_FUSED_CASE(7)
  }
#undef GWAS_FUSED_CASE
  c->launches++;
}
