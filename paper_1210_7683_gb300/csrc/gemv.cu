// Single-trait path of the mixed precision solve (t = 1): the contractions of Algorithm 5
// for one trait are matrix-vector products, so the pass is bound by HBM, not by the
// tensor cores.  One thread per SNP streams the SNP's resident operands (the exact
// genotypes and the three fixed-point slices of x'_c^2, 8 bytes per individual) once,
// 32 bytes per load, and forms the same exact-slice sums as the fused kernel's MMAs:
//   C1: x_i . [w1 | v_1..q | w2 | v_1..q | w3 | w4]  (slices of the trait's columns),
//   C2: [A1 A1 A1 A2 A2 A3s] . [E1 E2 E3s E2s E1 E1]  (slices of x'^2 against slices of e).
// Level-0 partial sums are integers below 2^24, so they are exact in FP32 in any order.
// The trait's slices (from the fused kernel's C1/C2 operands, trait 0 of tile 0) are held in
// shared memory as FP32 and read by broadcast.  The per-pair solve is the fused epilogue's.
#include <algorithm>
#include <cstdio>
#include <string>

#include "fused.cuh"
#include "gwas_internal.cuh"

namespace {

constexpr int GEMV_THREADS = 512;
constexpr int GEMV_KMAX = 2048;  // Kpad up to which the trait's rows fit shared memory

__device__ __forceinline__ void bf16x8(const uint4& v, float* f) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

template <int Q>
__global__ void __launch_bounds__(GEMV_THREADS, 1)
    gemv1_kernel(const __nv_bfloat16* __restrict__ G, const __nv_bfloat16* __restrict__ A2,
                 const __nv_bfloat16* __restrict__ B1, const __nv_bfloat16* __restrict__ B2, FusedArgs a) {
  constexpr int PM1 = Q, Q1 = Q > 0 ? Q : 1, TT = mixed_tt(Q), G1 = c1_groups(Q), NR = G1 + 4, CSTR = cst_stride(Q);
  constexpr int NRP = (NR + 3) / 4 * 4;  // row pitch: 16-byte aligned rows for vector loads
  extern __shared__ float4 trow4[];
  float* trow = (float*)trow4;  // [Kpad][NRP]: the trait's C1 groups, then E2s, E1, E2, E3s
  __shared__ float cj[CSTR];
  const int Kpad = a.Kpad;
  for (int idx = threadIdx.x; idx < NR * Kpad; idx += blockDim.x) {
    const int r = idx / Kpad, k = idx % Kpad;
    const __nv_bfloat16 v = r < G1 ? B1[(size_t)(r * TT) * Kpad + k] : B2[(size_t)((r - G1) * TT) * Kpad + k];
    trow[k * NRP + r] = __bfloat162float(v);
  }
  for (int e = threadIdx.x; e < CSTR; e += blockDim.x) cj[e] = a.cst[e];
  __syncthreads();
  const float inv_dof = 1.f / a.dof, F = 1.f / 256.f;
  const int64_t snp_end = a.row0 + a.nsnp;
  const int full_b = a.full_b;
  unsigned long long nsing = 0;
  for (int64_t base = a.row0 + (int64_t)blockIdx.x * blockDim.x; base < snp_end; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t snp = base + threadIdx.x;
    const bool valid = snp >= a.snp_lo && snp < snp_end;
    float acc[G1], c2[6];
#pragma unroll
    for (int r = 0; r < G1; ++r) acc[r] = 0.f;
#pragma unroll
    for (int r = 0; r < 6; ++r) c2[r] = 0.f;
    if (valid) {
      const uint4* g = (const uint4*)(G + (size_t)snp * Kpad);
      const uint4* p0 = (const uint4*)(A2 + (size_t)a2_row(0, snp) * Kpad);
      const uint4* p1 = (const uint4*)(A2 + (size_t)a2_row(1, snp) * Kpad);
      const uint4* p2 = (const uint4*)(A2 + (size_t)a2_row(2, snp) * Kpad);
      for (int k8 = 0; k8 < Kpad / 8; k8 += 2) {
        const uint4 gv[2] = {__ldg(g + k8), __ldg(g + k8 + 1)};
        const uint4 v0[2] = {__ldg(p0 + k8), __ldg(p0 + k8 + 1)};
        const uint4 v1[2] = {__ldg(p1 + k8), __ldg(p1 + k8 + 1)};
        const uint4 v2[2] = {__ldg(p2 + k8), __ldg(p2 + k8 + 1)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float xg[8], xa1[8], xa2[8], xa3[8];
          bf16x8(gv[h], xg);
          bf16x8(v0[h], xa1);
          bf16x8(v1[h], xa2);
          bf16x8(v2[h], xa3);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float* tr = trow + (size_t)(8 * (k8 + h) + e) * NRP;
#pragma unroll
            for (int r = 0; r < G1; ++r) acc[r] = fmaf(xg[e], tr[r], acc[r]);
            const float e2s = tr[G1], e1 = tr[G1 + 1], e2 = tr[G1 + 2], e3s = tr[G1 + 3];
            c2[0] = fmaf(xa1[e], e1, c2[0]);   // A1 x E1   (level 0)
            c2[1] = fmaf(xa1[e], e2, c2[1]);   // A1 x E2
            c2[2] = fmaf(xa1[e], e3s, c2[2]);  // A1 x E3s
            c2[3] = fmaf(xa2[e], e2s, c2[3]);  // A2 x E2s
            c2[4] = fmaf(xa2[e], e1, c2[4]);   // A2 x E1
            c2[5] = fmaf(xa3[e], e1, c2[5]);   // A3s x E1
          }
        }
      }
    }
    if (!valid) continue;
    // the fused kernel's epilogue for pair (snp, trait 0)
    const float sA = a.sA[snp];
    const float num = cj[0] * fmaf(F, fmaf(F, fmaf(F, acc[3 + 2 * PM1], acc[2 + 2 * PM1]), acc[1 + PM1]), acc[0]);
    float z[Q1], zz = 0.f;
#pragma unroll
    for (int c = 0; c < PM1; ++c) {
      z[c] = cj[1 + c] * fmaf(F, acc[2 + PM1 + c], acc[1 + c]);
      zz = fmaf(z[c], z[c], zz);
    }
    const float lvl1 = (c2[1] + c2[2]) + (c2[3] + c2[4]) + c2[5];
    const float s = (sA * cj[cst_escale(Q)]) * fmaf(F, lvl1, c2[0]);
    const float delta = s - zz;
    float beta, se;
    const bool sing = !(delta > 1e-6f * s) || !(sA > 0.f);
    if (sing) {
      beta = se = __int_as_float(0x7fc00000);
      ++nsing;
    } else {
      const float inv = __frcp_rn(delta);
      beta = num * inv;
      const float rss = fmaxf(fmaf(-num, beta, cj[cst_rr(Q)]), 0.f);
      se = __fsqrt_rn(rss * inv * inv_dof);
    }
    const int64_t o = snp - a.i0;
    if (full_b) {
      double* ob = a.out_b64 + o * (PM1 + 1);
#pragma unroll
      for (int c = 0; c < PM1; ++c) {
        // beta_L = g - L^-T z beta - a_i beta
        float t = cj[cst_g(Q) + c];
#pragma unroll
        for (int d = 0; d < PM1; ++d) t = fmaf(-cj[cst_lit(Q) + c * PM1 + d] * z[d], beta, t);
        t = fmaf(-a.acoef[snp * PM1 + c], beta, t);
        ob[c] = sing ? (double)beta : (double)t;
      }
      ob[PM1] = (double)beta;
    } else {
      a.out_beta[o] = beta;
      a.out_se[o] = se;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nsing += __shfl_xor_sync(0xffffffffu, nsing, o);
  if ((threadIdx.x & 31) == 0 && nsing) atomicAdd(a.singular, nsing);
}

}  // namespace

bool gemv1_supported(int q, int Kpad) { return q >= 0 && q <= 7 && Kpad <= GEMV_KMAX; }

int launch_gemv1(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2) {
  if (a.nsnp <= 0) return GWAS_OK;
  if (!gemv1_supported(q, a.Kpad)) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "single-trait kernel: p-1 or n out of range");
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t blocks = std::min<int64_t>(nsm, (a.nsnp + GEMV_THREADS - 1) / GEMV_THREADS);
  cudaError_t e = cudaSuccess;
  ProfScope ps(c, "gemv1");
  Q_DISPATCH(q, {
    auto kern = gemv1_kernel<Q>;
    const size_t smem = sizeof(float) * ((c1_groups(Q) + 4 + 3) / 4 * 4) * a.Kpad;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)blocks, GEMV_THREADS, smem, c->stream>>>(G, A2, B1, B2, a);
    e = cudaGetLastError();
  });
  c->launches++;
  if (e != cudaSuccess) return ctx_fail(c, GWAS_ERR_CUDA, std::string("single-trait kernel launch: ") + cudaGetErrorString(e));
  return GWAS_OK;
}
