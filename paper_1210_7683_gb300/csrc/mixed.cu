// Mixed-precision path of Algorithm 5: exact fixed-point slices of the operands on
// the bf16 tensor cores (FP32 accumulation), FP64 for the eigendecomposition and
// the per-trait algebra (S_TL, its Cholesky factor, g, the residual r_j).
//
// Resident data (per loaded genotype set):
//   G   [mpad][Kpad] bf16  exact genotypes x_i
//   G4  [mpad][Kp4 / 2]     the same as packed e2m1 pairs (when every value is one of e2m1's
//                             integers), the A operand of the CTA-pair kernel on e2m1 operands
//   A2  [mpad/128][3][128][Kpad] bf16  slices of x'_c^2 (a2_row), x'_c = Z^T P_c x_i (P_c: projector onto
//                             the complement of span(X_L), applied through the B operand)
//   sA  [m] float            per-SNP scale of the slices (0 for SNPs in span(X_L))
//   acoef [m][q] float       a_i with P_c x_i = x_i - X_L a_i (full coefficient output), q = p - 1
// Per gwas_solve trait block: Y' = Z^T Y and the back-rotated per-trait columns
//   w_j = M_j^-1 r_j and v'_j = P_c M_j^-1 X_L L_j^-T, both by exact sliced GEMMs.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fused.cuh"
#include "gwas_internal.cuh"
#include "xgemm.cuh"

struct MixedState {
  int Kpad = 0, bits = 0, ldx = 0;
  __nv_bfloat16 *Brot = nullptr, *Bzt = nullptr, *Bz = nullptr;  // B planes of the three rotations
  double *sBrot = nullptr, *sBzt = nullptr, *sBz = nullptr;       // their row scales
  double* XtXinv = nullptr;                                       // (X_L^T X_L)^-1 on the device
  int64_t m = 0, mpad = 0;
  __nv_bfloat16 *G = nullptr, *A2 = nullptr;
  int Kp4 = 0;             // padded n of the e2m1 operands (multiple of 256)
  uint8_t* G4 = nullptr;   // e2m1 genotypes, or NULL
  int* g4_bad = nullptr;   // device flag: a genotype outside e2m1's integers
  bool g4_ok = false;      // G4 holds the loaded genotypes exactly
  float *sA = nullptr, *acoef = nullptr;
  float* Xc = nullptr;     // FP32 scratch of the rotation, kept while slabs are reloaded
  int64_t xc_rows = 0;
  double* rk = nullptr;    // [n] ||P_c z_k||^2: the share of eigenvector k outside span(X_L)
  int64_t load_gen = 0;    // incremented by every genotype load (or slab)
  // S_BR by Chebyshev interpolation in h^2 (see the section at the end of this file)
  struct Cheb {
    int state = 0;               // 1: usable for h2_gen; -1: the exact contraction; 0: not planned
    int64_t h2_gen = -1;         // the context's heritability generation the plan was made for
    int R = 0;
    double lo = 0, hi = 1, bound = 0;
    MixedWs* ws = nullptr;       // operands of the R node heritabilities
    double* nodes = nullptr;     // [R]
    double* yzero = nullptr;     // [R][n] zero traits for the node operands
    double* tab = nullptr;       // [R][R] DCT weights
    float* T = nullptr;          // [t][CHEB_MAX_R] T_k(x_j) of the context's traits
    float* raw = nullptr;        // [2][R][ld] level-0 and level-1 node sums
    float* coef = nullptr;       // [CHEB_MAX_R + 1][ld] coefficients (last row: low part of c_0)
    int64_t ld = 0;              // columns of raw and coef
    int64_t coef_gen = -1;       // load generation the coefficients belong to
  } cheb;
};

// Eigen-directions k with ||P_c z_k||^2 at or below this carry no energy of any centred SNP
// (x'_c,k = (P_c z_k)^T x): their weights e_k are left out of the C2 operand and of its
// scale.  Typical case: a standardised kinship has the intercept as an eigenvector with a
// tiny eigenvalue, whose weight 1/(h^2 lambda + 1 - h^2) dominates as h^2 -> 1.
constexpr double RK_NULL = 1e-16;

static int cheb_coefficients(gwas_ctx* c);

// An allocation the caller can do without: on failure the context's last error is left as it was.
static bool try_alloc(gwas_ctx* c, size_t bytes, void** out) {
  const std::string saved = c->err;
  if (ctx_alloc(c, bytes, out) == GWAS_OK) return true;
  c->err = saved;
  return false;
}

namespace {

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }


// Rows of the FP64 B operand of the genotype rotation: row k < n is P_c z_k (so that
// (P_c Z)^T x = Z^T P_c x); row n + a holds the map x -> a_i[a] = ((X_L^T X_L)^-1 X_L^T x)[a].
template <int Q>
__global__ void rot_b_kernel(const double* __restrict__ Zc, const double* __restrict__ XL,
                             const double* __restrict__ XtXinv, int n, double* __restrict__ out,
                             double* __restrict__ rk) {
  constexpr int PM1 = Q, Q1 = Q > 0 ? Q : 1;
  const int k = blockIdx.x;
  __shared__ double red[Q1][8];
  __shared__ double coef[Q1];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (k < n) {
    const double* z = Zc + (size_t)k * n;
    double u[Q1] = {};
    for (int l = threadIdx.x; l < n; l += blockDim.x)
      for (int a = 0; a < PM1; ++a) u[a] += XL[(size_t)a * n + l] * z[l];
    for (int a = 0; a < PM1; ++a) {
      double v = u[a];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[a][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < PM1) {
      double s[Q1];
      for (int a = 0; a < PM1; ++a) {
        s[a] = 0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) s[a] += red[a][w];
      }
      double cf = 0;
      for (int b = 0; b < PM1; ++b) cf += XtXinv[threadIdx.x * PM1 + b] * s[b];
      coef[threadIdx.x] = cf;
    }
    __syncthreads();
    double r2 = 0;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      double v = z[l];
      for (int a = 0; a < PM1; ++a) v -= XL[(size_t)a * n + l] * coef[a];
      out[(size_t)k * n + l] = v;
      r2 += v * v;
    }
    // ||P_c z_k||^2
    __shared__ double rr[8];
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if (lane == 0) rr[warp] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) v += rr[w];
      rk[k] = v;
    }
  } else {
    const int a = k - n;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      double v = 0;
      for (int b = 0; b < PM1; ++b) v += XtXinv[a * PM1 + b] * XL[(size_t)b * n + l];
      out[(size_t)k * n + l] = v;
    }
  }
}

__global__ void transpose_kernel(const double* __restrict__ in, int n, double* __restrict__ out) {
  __shared__ double t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y)
    if (x < n && y0 + dy < n) t[dy][threadIdx.x] = in[(size_t)(y0 + dy) * n + x];
  __syncthreads();
  const int ox = y0 + threadIdx.x, oy0 = blockIdx.x * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y)
    if (ox < n && oy0 + dy < n) out[(size_t)(oy0 + dy) * n + ox] = t[threadIdx.x][dy];
}

// e2m1 codes (bit 3 the sign; magnitudes 0, 0.5, 1, 1.5, 2, 3, 4, 6 are codes 0..7) of the integers
// -8..7, nibble x + 8 of the table; the bit x + 8 of the mask marks the integers without a code.
constexpr uint64_t kE2m1Codes = 0x07065420ACDE0F00ull;  // x = -8 .. 7 from the low nibble up
constexpr uint32_t kE2m1Bad = 0xA00Bu;                  // -8, -7, -5, 5, 7
// e2m1 code of an integer genotype; a value without one (not in {0, +-1, +-2, +-3, +-4, +-6})
// clears ok and codes as 0.
__device__ __forceinline__ uint32_t e2m1_of_int(int x, bool& ok) {
  const uint32_t u = (uint32_t)(x + 8);
  if (u > 15u || ((kE2m1Bad >> u) & 1u)) {
    ok = false;
    return 0u;
  }
  return (uint32_t)(kE2m1Codes >> (4 * u)) & 15u;
}
// e2m1 code of a slice digit d in [-4, 4]: magnitude a has code a + min(a, 2)
__device__ __forceinline__ uint32_t e2m1_of_digit(int d) {
  const uint32_t a = (uint32_t)(d < 0 ? -d : d);
  return (a + min(a, 2u)) | (d < 0 ? 8u : 0u);
}

// int8 genotypes [m][n] -> bf16 [mpad][Kpad] (zero padded), and with `copy` the int8 bytes again
// into copy [m][n] (X may then be host memory the device reads, read once).  With G4 also the
// packed e2m1 pairs [mpad][Kp4 / 2] (element 2k in the low nibble of byte k), setting *bad when a
// value has no e2m1 code.  One thread per 8 consecutive values of a row: an 8-byte load when the
// row's bytes allow it, one 16-byte store (and one 4-byte store of e2m1 codes).
__global__ void geno_bf16_kernel(const int8_t* __restrict__ X, int64_t m, int n, int64_t mpad, int Kpad,
                                 __nv_bfloat16* __restrict__ G, int8_t* __restrict__ copy, uint8_t* __restrict__ G4,
                                 int Kp4, int* __restrict__ bad) {
  const int per_row = (G4 ? Kp4 : Kpad) / 8;
  const int64_t total = mpad * (int64_t)per_row;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / per_row;
    const int k0 = (int)(e - i * per_row) * 8;
    float v[8];
    const int64_t src = i * (int64_t)n + k0;
    // 8-byte accesses only where both addresses allow them (a caller's device or host pointer
    // may start anywhere)
    if (i < m && k0 + 8 <= n && ((uintptr_t)(X + src) & 7) == 0 && (!copy || ((uintptr_t)(copy + src) & 7) == 0)) {
      const uint2 w = *reinterpret_cast<const uint2*>(X + src);
      if (copy) *reinterpret_cast<uint2*>(copy + src) = w;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[j] = (float)(int8_t)((w.x >> (8 * j)) & 0xffu);
        v[4 + j] = (float)(int8_t)((w.y >> (8 * j)) & 0xffu);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const bool in = i < m && k0 + j < n;
        const int8_t x = in ? X[src + j] : (int8_t)0;
        if (in && copy) copy[src + j] = x;
        v[j] = (float)x;
      }
    }
    if (k0 < Kpad) {
      uint32_t u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        u[j] = *reinterpret_cast<const uint32_t*>(&b);
      }
      *reinterpret_cast<uint4*>(G + i * Kpad + k0) = make_uint4(u[0], u[1], u[2], u[3]);
    }
    if (G4) {
      bool ok = true;
      uint32_t w = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) w |= e2m1_of_int((int)v[j], ok) << (4 * j);
      if (!ok) atomicOr(bad, 1);
      *reinterpret_cast<uint32_t*>(G4 + i * (Kp4 / 2) + k0 / 2) = w;
    }
  }
}

// One warp per SNP: slices of x'_c^2 (three 8-bit fixed-point slices, scale = max/256,
// doubled while the level-0 partial sums could reach 2^24) and the centring coefficients.
__global__ void a2_slice_kernel(const float* __restrict__ Xc, int ldx, const int8_t* __restrict__ X, int64_t row0,
                                int64_t rows, int n, int64_t mpad, int Kpad, __nv_bfloat16* __restrict__ A2,
                                float* __restrict__ sA, float* __restrict__ acoef, int q) {
  const int warps = blockDim.x / 32;
  const int64_t r = blockIdx.x * (int64_t)warps + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (r >= rows) return;
  const int64_t i = row0 + r;
  const float* x = Xc + r * ldx;
  float mx = 0.f, nc = 0.f, nx = 0.f;
  for (int k = lane; k < n; k += 32) {
    const float v = x[k];
    mx = fmaxf(mx, v * v);
    nc = fmaf(v, v, nc);
    const float g = (float)X[i * n + k];
    nx = fmaf(g, g, nx);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
    nx += __shfl_xor_sync(0xffffffffu, nx, o);
  }
  // a SNP (numerically) inside span(X_L) has no Schur complement: flag it with scale 0
  const bool singular = !(nc > 1e-9f * fmaxf(nx, 1.f)) || !(mx > 0.f);
  float s = singular ? 1.f : mx / 256.f;
  // keep sum_k q0_k * 256 <= 2^24 so that level-0 products are exact
  for (int attempt = 0; attempt < 8; ++attempt) {
    float sum = 0.f;
    const float inv = 1.f / s;
    for (int k = lane; k < n; k += 32) sum += rintf(x[k] * x[k] * inv);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (sum <= 65536.f) break;
    s *= 2.f;
  }
  const float inv = 1.f / s;
  for (int k = lane; k < Kpad; k += 32) {
    float q0 = 0.f, q1 = 0.f, q2 = 0.f;
    if (k < n && !singular) {
      const float t = x[k] * x[k] * inv;
      q0 = rintf(t);
      const float r1 = (t - q0) * 256.f;
      q1 = rintf(r1);
      q2 = rintf((r1 - q1) * 256.f);
    }
    A2[a2_row(0, i) * Kpad + k] = __float2bfloat16(q0);
    A2[a2_row(1, i) * Kpad + k] = __float2bfloat16(q1);
    A2[a2_row(2, i) * Kpad + k] = __float2bfloat16(q2 * (1.f / 256.f));
  }
  if (lane == 0) sA[i] = singular ? 0.f : s;
  if (lane < q) acoef[i * q + lane] = x[n + lane];
}

// Per-trait FP64 algebra (Algorithm 5, per-trait lines) with e_j = diag(D_j^-1):
//   S_TL = X'_L^T diag(e) X'_L, b_T = X'_L^T (e . y'), L L^T = S_TL, g = S_TL^-1 b_T,
//   r' = y' - X'_L g,  rr = r'^T diag(e) r',
//   rows of Wt: [e . r' | (e . X'_L) L^-T]  (rotated basis; back-rotated by Z later),
//   slices of e in the C2 operand layout [E2s | E1 | E2 | E3s].
template <int Q>
__global__ void __launch_bounds__(256) prep_mixed_kernel(const double* __restrict__ Yt, int ldy,
                                                         const double* __restrict__ h2, const double* __restrict__ lam,
                                                         const double* __restrict__ XLt, int n, int Kpad,
                                                         double* __restrict__ Wt, __nv_bfloat16* __restrict__ B2,
                                                         float* __restrict__ cst, const int* __restrict__ slot,
                                                         int pair, const double* __restrict__ rk) {
  constexpr int PM1 = Q, Q1 = Q > 0 ? Q : 1, TT = mixed_tt(Q);
  constexpr int NTRI = PM1 * (PM1 + 1) / 2;
  const int j = blockIdx.x;
  const double h = h2[j];
  const double* y = Yt + (size_t)j * ldy;
  __shared__ double red[8], sh_ent[NTRI + Q1];         // lower triangle of S_TL, then b_T
  __shared__ double sh_L[Q1 * Q1], sh_Li[Q1 * Q1];      // L (lower) and L^-1 (lower), row-major
  __shared__ double sh_g[Q1], sh_Lit[Q1 * Q1], sh_se;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  // e_j, held in row 0 of this trait's Wt until w_j replaces it below, and its maximum
  double* e_row = Wt + (size_t)j * (PM1 + 1) * Kpad;
  double emax = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double e = 1.0 / (h * lam[k] + (1.0 - h));
    e_row[k] = e;
    if (rk[k] > RK_NULL) emax = fmax(emax, e);  // the C2 scale: directions SNPs can reach
  }
  for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (lane == 0) red[warp] = emax;
  __syncthreads();  // e_row (global) and red are visible to the whole block
  // S_TL = X'_L^T diag(e) X'_L (lower triangle) and b_T = X'_L^T (e . y'): a warp per entry
  for (int q = warp; q < NTRI + PM1; q += nw) {
    const double *u, *v;
    if (q < NTRI) {
      int a = 0;
      while ((a + 1) * (a + 2) / 2 <= q) ++a;
      u = XLt + (size_t)a * n;
      v = XLt + (size_t)(q - a * (a + 1) / 2) * n;
    } else {
      u = XLt + (size_t)(q - NTRI) * n;
      v = y;
    }
    double acc = 0;
    for (int k = lane; k < n; k += 32) acc = fma(e_row[k] * u[k], v[k], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh_ent[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double em = 0;
    for (int w = 0; w < nw; ++w) em = fmax(em, red[w]);
    // L L^T = S_TL
    for (int a = 0; a < PM1; ++a)
      for (int b = 0; b < PM1; ++b) {
        double v = 0;
        if (b <= a) {
          v = sh_ent[a * (a + 1) / 2 + b];
          for (int k = 0; k < b; ++k) v -= sh_L[a * Q1 + k] * sh_L[b * Q1 + k];
          v = (a == b) ? sqrt(fmax(v, 1e-300)) : v / sh_L[b * Q1 + b];
        }
        sh_L[a * Q1 + b] = v;
      }
    // L^-1 (lower)
    for (int c = 0; c < PM1; ++c)
      for (int a = 0; a < PM1; ++a) {
        double v = (a == c) ? 1.0 : 0.0;
        for (int k = 0; k < a; ++k) v -= sh_L[a * Q1 + k] * sh_Li[k * Q1 + c];
        sh_Li[a * Q1 + c] = v / sh_L[a * Q1 + a];
      }
    // g = L^-T L^-1 b_T; L^-1 b_T replaces b_T in place, last row first (row a reads rows <= a)
    for (int a = PM1 - 1; a >= 0; --a) {
      double v = 0;
      for (int k = 0; k <= a; ++k) v += sh_Li[a * Q1 + k] * sh_ent[NTRI + k];
      sh_ent[NTRI + a] = v;
    }
    for (int a = 0; a < PM1; ++a) {
      double v = 0;
      for (int k = a; k < PM1; ++k) v += sh_Li[k * Q1 + a] * sh_ent[NTRI + k];
      sh_g[a] = v;
    }
    for (int a = 0; a < PM1; ++a)
      for (int c = 0; c < PM1; ++c) sh_Lit[a * PM1 + c] = sh_Li[c * Q1 + a];  // (L^-T)[a][c]
    sh_se = em / 256.0;
  }
  __syncthreads();
  const double se = sh_se, inv_se = 1.0 / se;
  double rr = 0;
  const int p = PM1 + 1;
  const int tile = slot ? slot[j / TT] : j / TT, jj = j % TT;
  __nv_bfloat16* b2 = B2 + (size_t)tile * (pair ? c2_alloc(Q) : c2_rows(Q)) * Kpad;
  // rows of the four slices of e in the C2 operand of the tile:
  //   one CTA:   [E2s | E1 | E2 | E3s], 32 rows each;
  //   CTA pair:  each MMA's rows split between the two CTAs (E1 appears three times)
  int r_e2s, r_e1a, r_e1b, r_e1c, r_e2, r_e3s;
  if (!pair) {
    r_e2s = jj; r_e1a = TT + jj; r_e2 = 2 * TT + jj; r_e3s = 3 * TT + jj; r_e1b = r_e1c = -1;
  } else {
    r_e1a = jj; r_e2 = jj < TT / 2 ? TT + jj : 3 * TT + (jj - TT / 2);
    r_e2s = 3 * TT / 2 + jj; r_e1c = jj < TT / 2 ? 5 * TT / 2 + jj : 11 * TT / 2 + (jj - TT / 2);
    r_e3s = 7 * TT / 2 + jj; r_e1b = 9 * TT / 2 + jj;
  }
  for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
    double w = 0, v[Q1] = {};
    float q0 = 0, q1 = 0, q2 = 0;
    if (k < n) {
      const double e = e_row[k];  // from the first pass (this thread's k); w replaces it below
      double xl[Q1];
      for (int a = 0; a < PM1; ++a) xl[a] = XLt[(size_t)a * n + k];
      double r = y[k];
      for (int a = 0; a < PM1; ++a) r -= xl[a] * sh_g[a];
      w = e * r;
      rr += e * r * r;
      for (int c = 0; c < PM1; ++c) {
        double t = 0;
        for (int a = 0; a < PM1; ++a) t += xl[a] * sh_Lit[a * PM1 + c];
        v[c] = e * t;
      }
      const double t = rk[k] > RK_NULL ? e * inv_se : 0.0;
      const double d0 = rint(t);
      const double r1 = (t - d0) * 256.0;
      const double d1 = rint(r1);
      q0 = (float)d0;
      q1 = (float)d1;
      q2 = (float)rint((r1 - d1) * 256.0);
    }
    Wt[((size_t)j * p + 0) * Kpad + k] = w;
    for (int c = 0; c < PM1; ++c) Wt[((size_t)j * p + 1 + c) * Kpad + k] = v[c];
    b2[(size_t)r_e2s * Kpad + k] = __float2bfloat16(q1 * (1.f / 256.f));
    b2[(size_t)r_e1a * Kpad + k] = __float2bfloat16(q0);
    if (r_e1b >= 0) {
      b2[(size_t)r_e1b * Kpad + k] = __float2bfloat16(q0);
      b2[(size_t)r_e1c * Kpad + k] = __float2bfloat16(q0);
    }
    b2[(size_t)r_e2 * Kpad + k] = __float2bfloat16(q1);
    b2[(size_t)r_e3s * Kpad + k] = __float2bfloat16(q2 * (1.f / 256.f));
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  __syncthreads();
  if (lane == 0) red[warp] = rr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int w = 0; w < nw; ++w) v += red[w];
    float* cj = cst + ((size_t)tile * TT + jj) * cst_stride(Q);
    cj[cst_escale(Q)] = (float)se;
    cj[cst_rr(Q)] = (float)v;
    for (int a = 0; a < PM1; ++a) cj[cst_g(Q) + a] = (float)sh_g[a];
    for (int q = 0; q < PM1 * PM1; ++q) cj[cst_lit(Q) + q] = (float)sh_Lit[q];
  }
}

// Per trait: project the back-rotated columns [w | v_1..q] with P_c and write their
// fixed-point slices in the C1 operand layout (w: 4 slices, v: 2 slices).  With B1_4 (q = 3, the
// interpolated kernel's 24-trait tiles in the one-CTA order) the slices go there instead, as e2m1
// digits: slice digit q = 64 d0 + 8 d1 + d2 (|q| <= 256, so every d is in [-4, 4]), digit plane d
// of row r of a tile at [tile][r / 120][d][r % 120][Kp4 / 2], element 2k in the low nibble of byte k.
template <int Q>
__global__ void __launch_bounds__(256) pack_c1_kernel(const double* __restrict__ W, const double* __restrict__ XL,
                                                      const double* __restrict__ XtXinv, int n, int Kpad,
                                                      __nv_bfloat16* __restrict__ B1, float* __restrict__ cst,
                                                      const int* __restrict__ slot, int pair, int TT,
                                                      uint8_t* __restrict__ B1_4, int Kp4) {
  constexpr int PM1 = Q, Q1 = Q > 0 ? Q : 1;
  const int j = blockIdx.x;
  const int p = PM1 + 1;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  __shared__ double red[8][PM1 + 1];
  __shared__ double coef[Q1], smax;
  // TT: the trait-tile width of the layout (mixed_tt(Q), or tile_traits(Q, true) for the kernel
  // with S_BR interpolated); tiles of the C1 operand are c1_groups(Q) x TT rows
  const int tile = slot ? slot[j / TT] : j / TT, jj = j % TT;
  __nv_bfloat16* b1 = B1 + (size_t)tile * c1_groups(Q) * TT * Kpad;
  for (int c = 0; c < p; ++c) {
    const double* col = W + ((size_t)j * p + c) * Kpad;
    double u[Q1] = {};
    for (int l = threadIdx.x; l < n; l += blockDim.x)
      for (int a = 0; a < PM1; ++a) u[a] += XL[(size_t)a * n + l] * col[l];
    for (int a = 0; a < PM1; ++a) {
      double v = u[a];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][a] = v;
    }
    __syncthreads();
    if (threadIdx.x < PM1) {
      double s[Q1];
      for (int a = 0; a < PM1; ++a) {
        s[a] = 0;
        for (int w = 0; w < nw; ++w) s[a] += red[w][a];
      }
      double cf = 0;
      for (int b = 0; b < PM1; ++b) cf += XtXinv[threadIdx.x * PM1 + b] * s[b];
      coef[threadIdx.x] = cf;
    }
    __syncthreads();
    double mx = 0;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      double v = col[l];
      for (int a = 0; a < PM1; ++a) v -= XL[(size_t)a * n + l] * coef[a];
      mx = fmax(mx, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp][PM1] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0;
      for (int w = 0; w < nw; ++w) v = fmax(v, red[w][PM1]);
      smax = v > 0 ? v / 256.0 : 1.0;
      cst[((size_t)tile * TT + jj) * cst_stride(Q) + c] = (float)smax;
    }
    __syncthreads();
    const double inv = 1.0 / smax;
    const int nsl = c == 0 ? 4 : 2;
    // Digits below the first: w: three of 8 bits; v': one of 9 bits (|q| <= 256 is exact in bf16
    // and 2 * 256 * n stays below 2^24), which halves z's truncation error.  They come from one
    // 64-bit fixed-point integer per element, X = round(t * 2^fb) with fb = 24 (w) or 9 (v'), each
    // digit the rounded quotient of the remainder by the next power of two: the digits of rounding
    // digit by digit, with two FP64 operations for all of them instead of three per digit.
    const int fb = c == 0 ? 24 : 9, db = c == 0 ? 8 : 9;
    const double sc = ldexp(inv, fb);
    if (B1_4) {
      const int half_rows = c1_rows_of(3, true) / 2;
      const size_t rb = (size_t)Kp4 / 2;
      for (int l2 = threadIdx.x; l2 < Kp4 / 2; l2 += blockDim.x) {
        long long X2[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int l = 2 * l2 + e;
          double t = 0;
          if (l < n) {
            t = col[l];
            for (int a = 0; a < PM1; ++a) t -= XL[(size_t)a * n + l] * coef[a];
          }
          X2[e] = __double2ll_rn(t * sc);
        }
        for (int s = 0; s < nsl; ++s) {
          const int sh = fb - (s == 0 ? 0 : s * db);
          uint32_t code[3] = {0u, 0u, 0u};
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const long long q = sh > 0 ? ((X2[e] + (1LL << (sh - 1))) >> sh) : X2[e];
            X2[e] -= q * (1LL << sh);
            // |q| <= 256: every digit is in [-4, 4]
            const int qi = (int)q, d0 = (qi + 32) >> 6, r = qi - 64 * d0, d1 = (r + 4) >> 3, d2 = r - 8 * d1;
            code[0] |= e2m1_of_digit(d0) << (4 * e);
            code[1] |= e2m1_of_digit(d1) << (4 * e);
            code[2] |= e2m1_of_digit(d2) << (4 * e);
          }
          const int row = (s < 2 ? s * (1 + Q) + c : 2 * Q + s) * TT + jj;  // one-CTA order
          const int hf = row / half_rows, rr = row % half_rows;
#pragma unroll
          for (int d = 0; d < 3; ++d)
            B1_4[((((size_t)tile * 2 + hf) * 3 + d) * half_rows + rr) * rb + l2] = (uint8_t)code[d];
        }
      }
      __syncthreads();
      continue;
    }
    for (int l = threadIdx.x; l < Kpad; l += blockDim.x) {
      double t = 0;
      if (l < n) {
        t = col[l];
        for (int a = 0; a < PM1; ++a) t -= XL[(size_t)a * n + l] * coef[a];
      }
      long long X = __double2ll_rn(t * sc);  // |t * inv| <= 256: |X| <= 2^32
      for (int s = 0; s < nsl; ++s) {
        const int sh = fb - (s == 0 ? 0 : s * db);
        const long long q = sh > 0 ? ((X + (1LL << (sh - 1))) >> sh) : X;
        X -= q * (1LL << sh);
        // one CTA: groups [slice 1 of w, v_1..q | slice 2 of w, v_1..q | w3 | w4];
        // CTA pair (q = 3): [Q1 | Q3] for the first CTA, [Q2 | Q4] for the second
        int row;
        if (!pair) row = (s < 2 ? s * (1 + Q) + c : 2 * Q + s) * TT + jj;
        else row = (s == 0 ? 0 : s == 1 ? 5 * TT : s == 2 ? 4 * TT : 9 * TT) + (s < 2 ? c * TT : 0) + jj;
        b1[(size_t)row * Kpad + l] = __float2bfloat16_rn((float)(int)q);
      }
    }
    __syncthreads();
  }
}

}  // namespace

int64_t mixed_mpad(gwas_ctx* c) { return c->mixed ? c->mixed->mpad : 0; }
int mixed_kpad(gwas_ctx* c) { return c->mixed ? c->mixed->Kpad : 0; }
const float* mixed_sA(gwas_ctx* c) { return c->mixed ? c->mixed->sA : nullptr; }
const float* mixed_acoef(gwas_ctx* c) { return c->mixed ? c->mixed->acoef : nullptr; }
const __nv_bfloat16* mixed_G(gwas_ctx* c) { return c->mixed ? c->mixed->G : nullptr; }
const __nv_bfloat16* mixed_A2(gwas_ctx* c) { return c->mixed ? c->mixed->A2 : nullptr; }
int mixed_fp4_ready(gwas_ctx* c) { return c->mixed && c->mixed->G4 && c->mixed->g4_ok ? 1 : 0; }

void mixed_destroy(gwas_ctx* c) {
  if (!c->mixed) return;
  if (c->mixed->cheb.ws) mixed_ws_free(c, c->mixed->cheb.ws);
  delete c->mixed;
  c->mixed = nullptr;
}

void mixed_free(gwas_ctx* c) {
  MixedState* s = c->mixed;
  if (!s) return;
  ctx_free(c, s->G);
  ctx_free(c, s->A2);
  ctx_free(c, s->sA);
  ctx_free(c, s->acoef);
  ctx_free(c, s->Xc);
  ctx_free(c, s->G4);
  ctx_free(c, s->g4_bad);
  s->G4 = nullptr;
  s->g4_bad = nullptr;
  s->g4_ok = false;
  s->G = s->A2 = nullptr;
  s->sA = s->acoef = s->Xc = nullptr;
  s->m = s->mpad = s->xc_rows = 0;
}

static void mixed_destroy_setup(gwas_ctx* c) {
  MixedState* s = c->mixed;
  if (!s) return;
  ctx_free(c, s->Brot); ctx_free(c, s->Bzt); ctx_free(c, s->Bz);
  ctx_free(c, s->sBrot); ctx_free(c, s->sBzt); ctx_free(c, s->sBz);
  ctx_free(c, s->XtXinv);
  ctx_free(c, s->rk);
  s->rk = nullptr;
}

// One-time preparation of the B operands of the three rotations.
static int mixed_setup(gwas_ctx* c) {
  if (c->mixed && c->mixed->Brot) return GWAS_OK;
  if (c->pm1 < 0 || c->pm1 > MIXED_MAX_Q) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "mixed path needs 0 <= p-1 <= 19");
  if (!c->mixed) c->mixed = new MixedState;
  MixedState* s = c->mixed;
  const int n = c->n, PM1 = c->pm1;
  s->Kpad = (int)rup(n, 64);
  s->Kp4 = (int)rup(n, 256);
  s->bits = xgemm_bits(s->Kpad);
  s->ldx = (int)rup(n + PM1, 64);
  int rc;
  double *rot = nullptr, *zr = nullptr;
  const size_t plane_rows_rot = (size_t)s->ldx, plane_rows_z = (size_t)s->Kpad;
  if ((rc = ctx_alloc(c, sizeof(double) * std::max(1, PM1 * PM1), (void**)&s->XtXinv)) ||
      (rc = ctx_alloc(c, sizeof(double) * (size_t)(n + PM1) * n, (void**)&rot)) ||
      (rc = ctx_alloc(c, sizeof(double) * (size_t)n * n, (void**)&zr)) ||
      (rc = ctx_alloc(c, 2ull * 4 * plane_rows_rot * s->Kpad, (void**)&s->Brot)) ||
      (rc = ctx_alloc(c, 2ull * 4 * plane_rows_z * s->Kpad, (void**)&s->Bzt)) ||
      (rc = ctx_alloc(c, 2ull * 4 * plane_rows_z * s->Kpad, (void**)&s->Bz)) ||
      (rc = ctx_alloc(c, sizeof(double) * plane_rows_rot, (void**)&s->sBrot)) ||
      (rc = ctx_alloc(c, sizeof(double) * plane_rows_z, (void**)&s->sBzt)) ||
      (rc = ctx_alloc(c, sizeof(double) * plane_rows_z, (void**)&s->sBz)) ||
      (rc = ctx_alloc(c, sizeof(double) * n, (void**)&s->rk))) {
    ctx_free(c, rot);
    ctx_free(c, zr);
    mixed_destroy_setup(c);
    return rc;
  }
  if (PM1 > 0)
    cudaMemcpyAsync(s->XtXinv, c->h_XtXinv.data(), sizeof(double) * PM1 * PM1, cudaMemcpyHostToDevice, c->stream);
  { ProfScope ps(c, "setup_rotation_operands");
  Q_DISPATCH_ALL(PM1, rot_b_kernel<Q><<<n + PM1, 256, 0, c->stream>>>(c->Z, c->XL, s->XtXinv, n, rot, s->rk));
  c->launches++;
  dim3 tb(32, 8), tg((n + 31) / 32, (n + 31) / 32);
  transpose_kernel<<<tg, tb, 0, c->stream>>>(c->Z, n, zr);
  c->launches++; }
  launch_slice_rows(c, rot, n, n + PM1, n, s->ldx, s->Kpad, 4, s->bits, s->Brot, s->sBrot);
  launch_slice_rows(c, c->Z, n, n, n, s->Kpad, s->Kpad, 4, s->bits, s->Bzt, s->sBzt);
  launch_slice_rows(c, zr, n, n, n, s->Kpad, s->Kpad, 4, s->bits, s->Bz, s->sBz);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  ctx_free(c, rot);
  ctx_free(c, zr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, GWAS_ERR_CUDA, std::string("mixed setup: ") + cudaGetErrorString(e));
  }
  return GWAS_OK;
}

int mixed_load(gwas_ctx* c, const int8_t* dXR, int64_t m, bool reuse, int8_t* copy) {
  int rc = mixed_setup(c);
  if (rc) return rc;
  MixedState* s = c->mixed;
  const int n = c->n, PM1 = c->pm1;
  // a slab reuses the arrays when they hold enough rows (rows past m keep stale values,
  // which the fused kernel never writes out)
  // The e2m1 copy of the genotypes, for the CTA-pair kernel on e2m1 operands (p = 4), on a
  // one-time load.  Left out under GWAS_FP4=0, and in a context with an HBM budget: the copy and
  // the trait digits are memory such a budget did not account for, and an optional buffer held
  // from here could take the room a later call needs.
  const char* fp4_env = getenv("GWAS_FP4");
  const bool want_g4 = !reuse && PM1 == 3 && !(fp4_env && !strcmp(fp4_env, "0")) && c->budget == 0;
  if (!reuse || !s->G || s->mpad < rup(m, 128)) {
    mixed_free(c);
    s->mpad = rup(m, 128);
    if ((rc = ctx_alloc(c, 2ull * s->mpad * s->Kpad, (void**)&s->G)) ||
        (rc = ctx_alloc(c, 2ull * 3 * s->mpad * s->Kpad, (void**)&s->A2)) ||
        (rc = ctx_alloc(c, sizeof(float) * s->mpad, (void**)&s->sA)) ||
        (rc = ctx_alloc(c, sizeof(float) * s->mpad * std::max(1, PM1), (void**)&s->acoef))) {
      mixed_free(c);
      return rc;
    }
    // the e2m1 copy is optional: without room for it the bf16 operands serve
    if (want_g4 && !try_alloc(c, (size_t)s->mpad * (s->Kp4 / 2), (void**)&s->G4)) s->G4 = nullptr;
    if (s->G4 && !try_alloc(c, sizeof(int), (void**)&s->g4_bad)) {
      ctx_free(c, s->G4);
      s->G4 = nullptr;
    }
  }
  s->g4_ok = false;
  ++s->load_gen;
  uint8_t* G4 = want_g4 ? s->G4 : nullptr;  // NULL when there was no room for it
  if (G4) cudaMemsetAsync(s->g4_bad, 0, sizeof(int), c->stream);
  { ProfScope ps(c, "genotypes_bf16");
  geno_bf16_kernel<<<16 * 152, 256, 0, c->stream>>>(dXR, m, n, s->mpad, s->Kpad, s->G, copy, G4, s->Kp4, s->g4_bad);
  c->launches++; }
  // the genotypes read by the later kernels: the device copy the conversion made, if any
  if (copy) dXR = copy;
  // rotate in chunks of SNPs to bound the FP32 scratch
  const int64_t chunk = std::min<int64_t>(s->mpad, 1 << 18);
  if (s->xc_rows < chunk) {
    ctx_free(c, s->Xc);
    s->Xc = nullptr;
    s->xc_rows = 0;
    if ((rc = ctx_alloc(c, sizeof(float) * chunk * s->ldx, (void**)&s->Xc))) {
      mixed_free(c);
      return rc;
    }
    s->xc_rows = chunk;
  }
  float* Xc = s->Xc;
  for (int64_t r0 = 0; r0 < m && rc == GWAS_OK; r0 += chunk) {
    const int64_t rows = std::min<int64_t>(chunk, m - r0);
    XgemmArgs g{};
    g.rows = (int)rows;
    g.cols = n + PM1;
    g.rowsA_pad = (int)rup(rows, 128);
    g.rowsB_pad = s->ldx;
    g.Kpad = s->Kpad;
    g.level_scale = std::ldexp(1.0, -s->bits);
    g.scaleA = nullptr;
    g.scaleB = s->sBrot;
    g.out32 = Xc;
    g.ldo = s->ldx;
    g.status = c->d_status;
    g.name = "xgemm_rotate_snps";
    // x'_c = (P_c Z)^T x  (Algorithm 5, X'_R := Z^T X_R, on the centred SNPs)
    rc = launch_xgemm(c, 1, 4, 3, g, s->G + r0 * s->Kpad, s->Brot);
    if (rc == GWAS_OK) {
      const int warps = 8;
      ProfScope ps(c, "slice_snp_squares");
      a2_slice_kernel<<<(unsigned)((rows + warps - 1) / warps), warps * 32, 0, c->stream>>>(
          Xc, s->ldx, dXR, r0, rows, n, s->mpad, s->Kpad, s->A2, s->sA, s->acoef, PM1);
      c->launches++;
    }
  }
  if (rc) {
    cudaStreamSynchronize(c->stream);
    mixed_free(c);
    return rc;
  }
  if (!reuse) {
    // a one-time load gives its scratch back
    cudaStreamSynchronize(c->stream);
    ctx_free(c, s->Xc);
    s->Xc = nullptr;
    s->xc_rows = 0;
    if (G4) {
      int bad = 1;
      s->g4_ok = cudaMemcpy(&bad, s->g4_bad, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && bad == 0;
      cudaGetLastError();
    }
  }
  s->m = m;
  return GWAS_OK;
}

struct MixedWs {
  int tb_max = 0;
  __nv_bfloat16 *Ysl = nullptr, *Wsl = nullptr, *B1 = nullptr, *B2 = nullptr;
  double *sY = nullptr, *Yt = nullptr, *Wt = nullptr, *sW = nullptr;
  float* cst = nullptr;
  uint8_t* B1_4 = nullptr;  // the C1 operand as e2m1 digits (allocated by the first block that uses it)
  bool fp4 = false;         // the last prepared block's C1 operand is in B1_4
};

void mixed_ws_free(gwas_ctx* c, MixedWs* w) {
  if (!w) return;
  void* ps[] = {w->Ysl, w->Wsl, w->B1, w->B2, w->sY, w->Yt, w->Wt, w->sW, w->cst, w->B1_4};
  for (void* q : ps) ctx_free(c, q);
  delete w;
}

// Work buffers of a trait block of up to tb_max traits, allocated once per gwas_solve.
int mixed_ws_alloc(gwas_ctx* c, int tb_max, MixedWs** out) {
  *out = nullptr;
  int rc = mixed_setup(c);  // the rotation operands (one-time); no genotypes needed
  if (rc) return rc;
  MixedState* s = c->mixed;
  const int q = c->pm1, p = q + 1, Kpad = s->Kpad, TT = mixed_tt(q);
  const int nt_tiles = (tb_max + TT - 1) / TT;
  const int nt_alloc = (nt_tiles + fused_trait_tile_multiple() - 1) / fused_trait_tile_multiple() *
                       fused_trait_tile_multiple();
  const int rowsY = (int)rup(tb_max, 128), rowsW = (int)rup((int64_t)tb_max * p, 128);
  MixedWs* w = new MixedWs;
  w->tb_max = tb_max;
  if ((rc = ctx_alloc(c, 2ull * 4 * rowsY * Kpad, (void**)&w->Ysl)) ||
      (rc = ctx_alloc(c, sizeof(double) * rowsY, (void**)&w->sY)) ||
      (rc = ctx_alloc(c, sizeof(double) * (size_t)tb_max * Kpad, (void**)&w->Yt)) ||
      (rc = ctx_alloc(c, sizeof(double) * (size_t)tb_max * p * Kpad, (void**)&w->Wt)) ||
      (rc = ctx_alloc(c, 2ull * 4 * rowsW * Kpad, (void**)&w->Wsl)) ||
      (rc = ctx_alloc(c, sizeof(double) * rowsW, (void**)&w->sW)) ||
      (rc = ctx_alloc(c, 2ull * (size_t)c1_alloc_rows(q, tb_max) * Kpad, (void**)&w->B1)) ||
      (rc = ctx_alloc(c, 2ull * (size_t)nt_alloc * c2_alloc(q) * Kpad, (void**)&w->B2)) ||
      (rc = ctx_alloc(c, sizeof(float) * (size_t)nt_tiles * TT * cst_stride(q), (void**)&w->cst))) {
    mixed_ws_free(c, w);
    return rc;
  }
  *out = w;
  return GWAS_OK;
}

int mixed_prep_traits(gwas_ctx* c, MixedWs* w, const double* dY, const double* h2, int tb, __nv_bfloat16* B1,
                      __nv_bfloat16* B2, float* cst, const int* slot, int pair, int tt, uint8_t* B1_4) {
  MixedState* s = c->mixed;
  if (!s || !s->Brot) return ctx_fail(c, GWAS_ERR_STATE, "mixed path not set up");
  if (tb > w->tb_max) return ctx_fail(c, GWAS_ERR_ARG, "trait block larger than its workspace");
  const int n = c->n, q = c->pm1, p = q + 1, Kpad = s->Kpad;
  const int rowsY = (int)rup(tb, 128), rowsW = (int)rup((int64_t)tb * p, 128);
  int rc = GWAS_OK;
  __nv_bfloat16 *Ysl = w->Ysl, *Wsl = w->Wsl;
  double *sY = w->sY, *Yt = w->Yt, *Wt = w->Wt, *sW = w->sW;
  // Y' := Z^T Y (Algorithm 5, gemm) as an exact sliced GEMM
  launch_slice_rows(c, dY, n, tb, n, rowsY, Kpad, 4, s->bits, Ysl, sY);
  XgemmArgs g{};
  g.rows = tb;
  g.cols = n;
  g.rowsA_pad = rowsY;
  g.rowsB_pad = Kpad;
  g.Kpad = Kpad;
  g.level_scale = std::ldexp(1.0, -s->bits);
  g.scaleA = sY;
  g.scaleB = s->sBzt;
  g.out64 = Yt;
  g.ldo = Kpad;
  g.status = c->d_status;
  g.name = "xgemm_rotate_traits";
  if ((rc = launch_xgemm(c, 4, 4, 3, g, Ysl, s->Bzt)) == GWAS_OK) {
    {
      // per-trait algebra and the C2 operand
      ProfScope ps(c, "prep_traits");
      Q_DISPATCH_ALL(q, prep_mixed_kernel<Q><<<tb, 256, 0, c->stream>>>(Yt, Kpad, h2, c->lam, c->XLt, n, Kpad, Wt, B2,
                                                                    cst, slot, pair, s->rk));
      c->launches++;
    }
    // back-rotation [w | v] = Z [e.r' | (e.X'_L) L^-T]
    launch_slice_rows(c, Wt, Kpad, tb * p, n, rowsW, Kpad, 4, s->bits, Wsl, sW);
    XgemmArgs b = g;
    b.rows = tb * p;
    b.cols = n;
    b.rowsA_pad = rowsW;
    b.scaleA = sW;
    b.scaleB = s->sBz;
    b.out64 = Wt;
    b.name = "xgemm_back_rotate";
    rc = launch_xgemm(c, 4, 4, 3, b, Wsl, s->Bz);
  }
  if (rc == GWAS_OK) {
    ProfScope ps(c, "pack_trait_columns");
    const int TTc = tt > 0 ? tt : mixed_tt(q);
    Q_DISPATCH_ALL(q, pack_c1_kernel<Q><<<tb, 256, 0, c->stream>>>(Wt, c->XL, s->XtXinv, n, Kpad, B1, cst, slot, pair,
                                                                    TTc, B1_4, s->Kp4));
    c->launches++;
  }
  return rc;
}

int mixed_prep_block(gwas_ctx* c, MixedWs* w, const double* dY, int j0, int tb) {
  MixedState* s = c->mixed;
  if (!s || !s->Brot) return ctx_fail(c, GWAS_ERR_STATE, "mixed path not set up");
  if (tb > w->tb_max) return ctx_fail(c, GWAS_ERR_ARG, "trait block larger than its workspace");
  const int q = c->pm1, Kpad = s->Kpad, TT = mixed_tt(q);
  const int nt_tiles = (tb + TT - 1) / TT;
  const int nt_alloc = (nt_tiles + fused_trait_tile_multiple() - 1) / fused_trait_tile_multiple() *
                       fused_trait_tile_multiple();
  // the trait operands in the layout of the kernel that will run: the interpolated kernel's
  // (its tile width, one-CTA order), or the contracting kernel's (pair order for the CTA pair);
  // the interpolated pair at p = 4 on genotypes with an e2m1 copy: e2m1 digits of the C1 slices
  const bool ip = mixed_block_interp(c, tb);
  w->fp4 = ip && q == 3 && mixed_pair_layout(c) && mixed_fp4_ready(c);
  if (w->fp4 && !w->B1_4) {
    // optional too: without room for the e2m1 digits the block runs on bf16 operands
    const size_t bytes = (size_t)((w->tb_max + 23) / 24 + 3) / 4 * 4 * FP4_TILE_ROWS * (s->Kp4 / 2);
    if (!try_alloc(c, bytes, (void**)&w->B1_4)) {
      w->B1_4 = nullptr;
      w->fp4 = false;
    }
  }
  if (w->fp4) {
    const size_t used = (size_t)((tb + 23) / 24 + 3) / 4 * 4 * FP4_TILE_ROWS * (s->Kp4 / 2);
    cudaMemsetAsync(w->B1_4, 0, used, c->stream);
  } else {
    cudaMemsetAsync(w->B1, 0, 2ull * c1_alloc_rows(q, tb) * Kpad, c->stream);
  }
  cudaMemsetAsync(w->B2, 0, 2ull * nt_alloc * c2_alloc(q) * Kpad, c->stream);
  return mixed_prep_traits(c, w, dY, c->h2 + j0, tb, w->B1, w->B2, w->cst, nullptr, ip ? 0 : mixed_pair_layout(c),
                           ip ? tile_traits(q, true) : 0, w->fp4 ? w->B1_4 : nullptr);
}

int mixed_fused_ops(gwas_ctx* c, const __nv_bfloat16* B1, const __nv_bfloat16* B2, const float* cst, int tb, int64_t i0,
                    int64_t i1, int64_t ldo, void* out, int j0, const uint8_t* B1_4) {
  MixedState* s = c->mixed;
  if (!s || !s->G) return ctx_fail(c, GWAS_ERR_STATE, "mixed genotypes not loaded");
  const int n = c->n, q = c->pm1, p = q + 1, Kpad = s->Kpad;
  // S_BR from its Chebyshev series in h^2 when the plan allows it (traits of the context)
  const bool interp = j0 >= 0 && mixed_block_interp(c, tb);
  const int TT = tile_traits(q, interp);
  const int nt_tiles = (tb + TT - 1) / TT;
  int rc = GWAS_OK;
  {
    FusedArgs a{};
    // tiles start on multiples of 128 SNPs; those below i0 are not written
    a.row0 = i0 & ~(int64_t)127;
    a.snp_lo = i0;
    a.i0 = i0;
    a.nsnp = i1 - a.row0;
    a.n_stiles = (int)((a.nsnp + 127) / 128);
    a.n_ttiles = nt_tiles;
    a.group = std::max(1, c->tune.group);
    if (const char* e = getenv("GWAS_FUSED_GROUP")) a.group = std::max(1, atoi(e));
    a.ntrait = tb;
    a.Kpad = Kpad;
    a.Kp4 = s->Kp4;
    a.mpad = s->mpad;
    a.dof = (float)(n - p);
    (void)n;
    a.sA = s->sA;
    a.acoef = s->acoef;
    a.cst = cst;
    a.full_b = c->output == GWAS_OUT_FULL_B;
    a.ldo = ldo;
    if (a.full_b) {
      a.out_b64 = (double*)out;
    } else {
      void** pr = (void**)out;
      a.out_beta = (float*)pr[0];
      a.out_se = (float*)pr[1];
    }
    a.status = c->d_status;
    a.singular = c->d_status + 1;
    const bool gemv = tb == 1 && gemv1_supported(q, Kpad) && !mixed_pair_layout(c);
    if (interp) {
      if ((rc = cheb_coefficients(c))) return rc;
      a.cheb_coef = s->cheb.coef;
      a.cheb_T = s->cheb.T + (size_t)j0 * CHEB_MAX_R;
      a.cheb_R = s->cheb.R;
      a.cheb_ld = s->cheb.ld;
    }
    // one trait: the contractions are matrix-vector products, bound by HBM (gemv.cu)
    if (B1_4) {
      // the C1 operand was prepared as e2m1 digits for the interpolated pair (mixed_prep_block)
      if (!interp || q != 3 || !mixed_pair_layout(c) || !mixed_fp4_ready(c))
        return ctx_fail(c, GWAS_ERR_STATE, "e2m1 trait operands without the kernel that reads them");
      if (a.n_stiles == 0 || a.n_ttiles == 0) return GWAS_OK;
      rc = launch_fused_cheb_pair_fp4(c, a, s->G4, B1_4, (a.n_ttiles + 3) / 4 * 4);
    } else if (gemv) rc = launch_gemv1(c, q, a, s->G, s->A2, B1, B2);
    else rc = launch_fused(c, q, a, s->G, s->A2, B1, B2);
  }
  return rc;
}

int mixed_fused_block(gwas_ctx* c, MixedWs* w, int tb, int64_t i0, int64_t i1, int64_t ldo, void* out, int j0) {
  return mixed_fused_ops(c, w->B1, w->B2, w->cst, tb, i0, i1, ldo, out, j0, w->fp4 ? w->B1_4 : nullptr);
}

int mixed_solve_block(gwas_ctx* c, MixedWs* w, const double* dY, int j0, int tb, int64_t i0, int64_t i1, int64_t ldo,
                      void* out) {
  int rc = mixed_prep_block(c, w, dY, j0, tb);
  return rc ? rc : mixed_fused_block(c, w, tb, i0, i1, ldo, out, j0);
}

// ---------------------------------------------------------------- S_BR by Chebyshev interpolation in h^2
//
// For SNP i, S_BR as a function of the heritability, s_i(h) = sum_k e_k(h) x'^2_ck with
// e_k(h) = 1 / (1 - h + h lambda_k), is a positive combination of the functions e_k.  On an
// interval [lo, hi] holding the context's heritabilities it is replaced by its interpolant at the
// R Chebyshev points of [lo, hi] (a polynomial of degree R - 1 in h):
//   - the node values s_i(h_r) are the exact contraction (X'_R o X'_R)^T D^-1 of the fused kernel
//     (Algorithm 5's S_BR) for R node heritabilities, taken from its level-0 and level-1 sums;
//   - their Chebyshev coefficients c_ik follow by a discrete cosine transform (FP64);
//   - the fused kernel then evaluates s_ij = sum_k c_ik T_k(x_j), x_j the image of h_j in [-1, 1],
//     instead of contracting the squares of the rotated SNPs with D_j^-1 for every trait.
// The interpolant of 1/(a + b h) with its pole at h* has relative error omega(h) / omega(h*) at h,
// omega the node polynomial, so that, the terms being positive, s_i has relative error at most
// max_k max_h |omega(h)| / |omega(h*_k)| over the eigen-directions that centred SNPs reach.  R is
// the least number of nodes with that bound <= kChebTol; when no R <= CHEB_MAX_R meets it (a pole
// close to the interval: an eigenvalue near 0 reached by the SNPs and heritabilities near 1), or
// GWAS_S_BR=exact is set, the fused kernel contracts S_BR itself.

namespace {

constexpr double kChebTol = 1e-10;

// T_k(x_j) for the context's traits, k < R (zero beyond)
__global__ void cheb_t_kernel(const double* __restrict__ h2, int t, double lo, double hi, int R, float* __restrict__ T) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= t) return;
  const double x = fmin(1.0, fmax(-1.0, (2.0 * h2[j] - (lo + hi)) / (hi - lo)));
  double tm = 1.0, tk = x;
  for (int k = 0; k < CHEB_MAX_R; ++k) {
    double v = 0.0;
    if (k == 0) v = 1.0;
    else if (k == 1) v = x;
    else {
      const double tn = 2.0 * x * tk - tm;
      tm = tk;
      tk = tn;
      v = tn;
    }
    T[(size_t)j * CHEB_MAX_R + k] = k < R ? (float)v : 0.f;
  }
}

// Coefficients of SNP i from its node sums: s_i(h_r) = sA_i escale_r (level 0 + level 1 / 256),
// c_k = sum_r tab[k][r] s_i(h_r) in FP64; c_0 is kept as two floats.
__global__ void __launch_bounds__(256) cheb_coef_kernel(const float* __restrict__ raw, int R, int64_t ld, int64_t m,
                                                        const float* __restrict__ sA, const float* __restrict__ cst,
                                                        int cstr, int eoff, const double* __restrict__ tab,
                                                        float* __restrict__ coef) {
  __shared__ double stab[CHEB_MAX_R * CHEB_MAX_R];
  __shared__ double sesc[CHEB_MAX_R];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) stab[e] = tab[e];
  for (int e = threadIdx.x; e < R; e += blockDim.x) sesc[e] = (double)cst[(size_t)e * cstr + eoff];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ld) return;
  // rows past m (tile padding) get zero coefficients; their node sums were never written
  double sv[CHEB_MAX_R];
  const bool in = i < m;
  const double a = in ? (double)sA[i] : 0.0;
#pragma unroll
  for (int r = 0; r < CHEB_MAX_R; ++r)
    sv[r] = (in && r < R)
                ? a * sesc[r] * ((double)raw[(size_t)r * ld + i] + (double)raw[(size_t)(R + r) * ld + i] * (1.0 / 256.0))
                : 0.0;
  for (int k = 0; k < R; ++k) {
    double ck = 0.0;
#pragma unroll
    for (int r = 0; r < CHEB_MAX_R; ++r)
      if (r < R) ck = fma(stab[k * R + r], sv[r], ck);
    const float hi = (float)ck;
    coef[(size_t)k * ld + i] = hi;
    if (k == 0) coef[(size_t)CHEB_MAX_R * ld + i] = (float)(ck - (double)hi);
  }
}

// The Chebyshev points of [lo, hi], largest first (x_r = cos(pi r / (R - 1))).
void cheb_nodes(int R, double lo, double hi, double* h) {
  for (int r = 0; r < R; ++r) h[r] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos(M_PI * r / (R - 1));
}

}  // namespace

// Relative error bound of the degree-(R-1) interpolant of every e_k on [lo, hi] (see above);
// reach[k] != 0 marks the eigen-directions that enter S_BR.
static double cheb_bound(int n, const double* lam, const unsigned char* reach, double lo, double hi, int R) {
  std::vector<double> h(R);
  cheb_nodes(R, lo, hi, h.data());
  // max |omega| over a fine grid of [lo, hi], with a margin for the grid.  Every factor is at most
  // hi - lo <= 1, so the products neither overflow nor, at their maximum (about
  // 2^(2-R) ((hi - lo) / 2)^R >= 1e-90), underflow; the loop over the grid vectorises.
  const int G = 4096;
  std::vector<double> w(G + 1, 1.0);
  for (int r = 0; r < R; ++r) {
    const double hr = h[r];
    for (int g = 0; g <= G; ++g) w[g] *= std::fabs(lo + (hi - lo) * g / G - hr) + 1e-300;
  }
  const double lmax = std::log(*std::max_element(w.begin(), w.end())) + std::log(2.0);
  // min over the reached k of log |omega(pole_k)|: factors in groups of 8 stay inside FP64's range
  // (each is between the distance of the pole to [lo, hi] and |pole| + 1 <= 2^53 + 1)
  double lmin = INFINITY;
  for (int k = 0; k < n; ++k) {
    if (!reach[k] || lam[k] == 1.0) continue;
    const double hs = 1.0 / (1.0 - lam[k]);   // the pole of 1 / (1 - h + h lambda_k)
    if (hs >= lo && hs <= hi) return INFINITY;
    double l = 0;
    for (int r0 = 0; r0 < R; r0 += 8) {
      double p = 1.0;
      for (int r = r0; r < std::min(R, r0 + 8); ++r) p *= std::fabs(hs - h[r]);
      l += std::log(p);
    }
    lmin = std::min(lmin, l);
  }
  return lmin == INFINITY ? 0.0 : std::exp(lmax - lmin);
}

extern "C" int gwas_cheb_plan(int n, const double* lam, const unsigned char* reach, double lo, double hi, double tol,
                              int* R, double* bound) {
  if (n < 1 || !lam || !reach || !R || !(lo >= 0.0) || !(hi <= 1.0) || !(hi > lo) || !(tol > 0.0)) return GWAS_ERR_ARG;
  *R = 0;
  double b = INFINITY;
  for (int r = 4; r <= CHEB_MAX_R; ++r) {
    b = cheb_bound(n, lam, reach, lo, hi, r);
    if (b <= tol) {
      *R = r;
      break;
    }
  }
  if (bound) *bound = b;
  return GWAS_OK;
}

int mixed_cheb_plan(gwas_ctx* c) {
  MixedState* s = c->mixed;
  if (!s || !s->rk || c->h_h2.empty()) return -1;
  auto& ch = s->cheb;
  if (ch.state != 0 && ch.h2_gen == c->h2_gen) return ch.state;
  ch.h2_gen = c->h2_gen;
  ch.state = -1;
  ch.coef_gen = -1;
  if (const char* e = getenv("GWAS_S_BR"))
    if (!strcmp(e, "exact")) return -1;
  const int n = c->n, t = (int)c->h_h2.size();  // every trait of the context (c->t may be a sample's)
  double lo = *std::min_element(c->h_h2.begin(), c->h_h2.end());
  double hi = *std::max_element(c->h_h2.begin(), c->h_h2.end());
  if (hi - lo < 1e-3) {  // a narrow interval: widen it, inside [0, 1]
    const double mid = std::min(1.0 - 5e-4, std::max(5e-4, 0.5 * (lo + hi)));
    lo = mid - 5e-4;
    hi = mid + 5e-4;
  }
  std::vector<double> rk(n);
  if (cudaMemcpy(rk.data(), s->rk, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  std::vector<unsigned char> reach(n);
  for (int k = 0; k < n; ++k) reach[k] = rk[k] > RK_NULL;
  int R = 0;
  double bound = 0;
  gwas_cheb_plan(n, c->h_lam.data(), reach.data(), lo, hi, kChebTol, &R, &bound);
  if (R == 0) return -1;
  // node operands (zero traits at the node heritabilities), DCT weights and T_k(x_j)
  if (!ch.ws) {
    if (mixed_ws_alloc(c, CHEB_MAX_R, &ch.ws) || ctx_alloc(c, sizeof(double) * CHEB_MAX_R, (void**)&ch.nodes) ||
        ctx_alloc(c, sizeof(double) * CHEB_MAX_R * n, (void**)&ch.yzero) ||
        ctx_alloc(c, sizeof(double) * CHEB_MAX_R * CHEB_MAX_R, (void**)&ch.tab) ||
        ctx_alloc(c, sizeof(float) * (size_t)t * CHEB_MAX_R, (void**)&ch.T)) {
      c->err.clear();
      return -1;
    }
    cudaMemsetAsync(ch.yzero, 0, sizeof(double) * CHEB_MAX_R * n, c->stream);
  }
  std::vector<double> h(R), tab((size_t)R * R);
  cheb_nodes(R, lo, hi, h.data());
  for (int k = 0; k < R; ++k)
    for (int r = 0; r < R; ++r) {
      const double w = (r == 0 || r == R - 1) ? 0.5 : 1.0, ck = (k == 0 || k == R - 1) ? 0.5 : 1.0;
      tab[(size_t)k * R + r] = 2.0 / (R - 1) * w * ck * std::cos(M_PI * k * r / (R - 1));
    }
  cudaMemcpyAsync(ch.nodes, h.data(), sizeof(double) * R, cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(ch.tab, tab.data(), sizeof(double) * R * R, cudaMemcpyHostToDevice, c->stream);
  const int q = c->pm1, Kpad = s->Kpad;
  const int nt_tiles = (CHEB_MAX_R + mixed_tt(q) - 1) / mixed_tt(q);
  const int nt_pad = (nt_tiles + fused_trait_tile_multiple() - 1) / fused_trait_tile_multiple() * fused_trait_tile_multiple();
  cudaMemsetAsync(ch.ws->B1, 0, 2ull * c1_alloc_rows(q, CHEB_MAX_R) * Kpad, c->stream);
  cudaMemsetAsync(ch.ws->B2, 0, 2ull * nt_pad * c2_alloc(q) * Kpad, c->stream);
  if (mixed_prep_traits(c, ch.ws, ch.yzero, ch.nodes, R, ch.ws->B1, ch.ws->B2, ch.ws->cst, nullptr, 0, 0)) {
    c->err.clear();
    return -1;
  }
  cheb_t_kernel<<<(t + 255) / 256, 256, 0, c->stream>>>(c->h2, t, lo, hi, R, ch.T);
  c->launches++;
  ch.R = R;
  ch.lo = lo;
  ch.hi = hi;
  ch.bound = bound;
  ch.state = 1;
  return 1;
}

int mixed_pair_layout(gwas_ctx* c) { return fused_pair_layout(c, c->pm1); }

bool mixed_block_interp(gwas_ctx* c, int tb) { return tb > 1 && mixed_cheb_plan(c) == 1; }

int mixed_cheb_info(gwas_ctx* c, int* R, double* lo, double* hi, double* bound) {
  const int st = c->mixed ? c->mixed->cheb.state : 0;
  if (st == 1) {
    *R = c->mixed->cheb.R;
    *lo = c->mixed->cheb.lo;
    *hi = c->mixed->cheb.hi;
    *bound = c->mixed->cheb.bound;
  } else {
    *R = 0;
    *lo = *hi = *bound = 0;
  }
  return st;
}

// The coefficients of the loaded SNPs (once per load): the exact kernel at the node heritabilities,
// then the transform.
static int cheb_coefficients(gwas_ctx* c) {
  MixedState* s = c->mixed;
  auto& ch = s->cheb;
  if (ch.coef_gen == s->load_gen) return GWAS_OK;
  const int q = c->pm1, R = ch.R;
  int rc;
  if (ch.ld < s->mpad) {
    ctx_free(c, ch.raw);
    ctx_free(c, ch.coef);
    ch.raw = ch.coef = nullptr;
    ch.ld = 0;
    if ((rc = ctx_alloc(c, sizeof(float) * 2 * CHEB_MAX_R * s->mpad, (void**)&ch.raw)) ||
        (rc = ctx_alloc(c, sizeof(float) * (CHEB_MAX_R + 1) * s->mpad, (void**)&ch.coef)))
      return rc;
    ch.ld = s->mpad;
  }
  FusedArgs a{};
  a.row0 = 0;
  a.snp_lo = 0;
  a.i0 = 0;
  a.nsnp = s->m;
  a.n_stiles = (int)((s->m + 127) / 128);
  a.n_ttiles = (R + mixed_tt(q) - 1) / mixed_tt(q);
  a.group = 16;
  a.ntrait = R;
  a.Kpad = s->Kpad;
  a.mpad = s->mpad;
  a.dof = (float)(c->n - c->p);
  a.sA = s->sA;
  a.acoef = s->acoef;
  a.cst = ch.ws->cst;
  a.full_b = 2;
  a.ldo = ch.ld;
  a.out_beta = ch.raw;
  a.out_se = ch.raw + (size_t)R * ch.ld;
  a.status = c->d_status;
  a.singular = c->d_status + 1;
  if ((rc = launch_fused(c, q, a, s->G, s->A2, ch.ws->B1, ch.ws->B2))) return rc;
  {
    ProfScope ps(c, "cheb_coefficients");
    cheb_coef_kernel<<<(unsigned)((ch.ld + 255) / 256), 256, 0, c->stream>>>(
        ch.raw, R, ch.ld, s->m, s->sA, ch.ws->cst, cst_stride(q), cst_escale(q), ch.tab, ch.coef);
    c->launches++;
  }
  ch.coef_gen = s->load_gen;
  return GWAS_OK;
}

extern "C" int gwas_sbr_info(gwas_ctx* c, int* terms, double* lo, double* hi, double* bound) {
  if (!c || !terms || !lo || !hi || !bound) return GWAS_ERR_ARG;
  if (c->precision != GWAS_MIXED || !c->mixed) {
    *terms = 0;
    *lo = *hi = *bound = 0;
    return GWAS_OK;
  }
  DeviceGuard guard(c->device);
  mixed_cheb_plan(c);
  mixed_cheb_info(c, terms, lo, hi, bound);
  return GWAS_OK;
}
