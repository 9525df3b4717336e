#pragma once
// Single-trait path of the mixed precision solve (t = 1): the contractions of Algorithm 5
// for one trait are matrix-vector products, so the pass is bound by HBM, not by the
// tensor cores.  Every SNP's resident operands (the exact genotypes and the three
// fixed-point slices of x'_c^2, 8 bytes per individual) are streamed once, and the same
// exact-slice sums as the fused kernel's MMAs are formed on the CUDA cores:
//   C1: x_i . [w1 | v_1..q | w2 | v_1..q | w3 | w4]  (slices of the trait's columns),
//   C2: [A1 A1 A1 A2 A2 A3s] . [E1 E2 E3s E2s E1 E1]  (slices of x'^2 against slices of e).
// Level-0 partial sums are integers below 2^24, so they are exact in FP32 in any order.
// The per-pair solve is the fused epilogue's.
//
// One persistent CTA per SM: a TMA producer warp and 4 consumer warps, 256 SNPs (two 128-SNP
// tiles) per unit, two SNPs per thread (row r of each tile), so that each read of the trait's
// slices from shared memory serves two SNPs (one SNP per thread on 8 warps for p - 1 >= 8).  A
// stage holds 32 values of k: eight 8 KB boxes
// (genotypes and the three planes, two tiles; 64-byte swizzle, so that the row-per-thread
// reads are free of bank conflicts) and the trait's 32-wide slices (two strided boxes that
// pick trait 0's row of every group).  A ring of three stages keeps ~200 KB per SM in flight.
#include <algorithm>
#include <cstdio>
#include <string>

#include "fused.cuh"
#include "gwas_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int GK = 32;                   // values of k per stage
constexpr int GNS = 3;                   // ring stages
constexpr int GUNIT = 256;               // SNPs per unit: two 128-row tiles
// Consumers: 4 warps with two SNPs per thread (row r of both tiles), so that every broadcast
// read of the trait's row serves two SNPs; for p - 1 >= 8 (up to 48 accumulators per SNP) 8 warps
// with one SNP per thread, which measured 2-6 % faster there (the shared-memory wavefronts of
// the broadcast reads bound the kernel at large p).
template <int Q>
struct GemvPar {
  static constexpr int NT = Q >= 8 ? 1 : 2;  // SNPs (tiles) per consumer thread
  static constexpr int THR = GUNIT / NT;     // consumer threads
  static constexpr int CONS = THR / 32;      // consumer warps
};
constexpr int GBOX = 128 * GK * 2;       // one box: 128 rows x 32 bf16 = 8 KB
constexpr int GDATA = 8 * GBOX;          // G + three planes, two tiles

template <int Q>
struct GemvGeo {
  // NRP: the FP32 row stride, = 2 (mod 4): the per-stage conversion writes consecutive k at
  // this stride, which then meets 16 banks (a multiple of 4 met 2 banks: 16-way conflicts);
  // the rows stay 8-byte aligned for the main loop's float2 broadcast reads
  static constexpr int G1 = c1_groups(Q), NR = G1 + 4, NRP = NR % 4 == 2 ? NR : NR + 2;
  static constexpr int TRAW = (NR * GK * 2 + 1023) / 1024 * 1024;  // bf16 trait rows of a stage
  static constexpr int STAGE = GDATA + TRAW;
  static constexpr int TF32 = GK * NRP * 4;                         // the same rows, FP32, [k][row]
  static constexpr int SMEM = GNS * STAGE + GNS * TF32 + 1024 + 256;
};

__device__ __forceinline__ void bf16x8(const uint4& v, float* f) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

template <int Q>
__global__ void __launch_bounds__(32 + GemvPar<Q>::THR, 1)
    gemv1_kernel(const __grid_constant__ CUtensorMap mapG, const __grid_constant__ CUtensorMap mapA,
                 const __grid_constant__ CUtensorMap mapT1, const __grid_constant__ CUtensorMap mapT2, FusedArgs a) {
  using Geo = GemvGeo<Q>;
  constexpr int PM1 = Q, Q1 = Q > 0 ? Q : 1, G1 = Geo::G1, NR = Geo::NR, NRP = Geo::NRP, CSTR = cst_stride(Q);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* tf = (float*)(smem + GNS * Geo::STAGE);  // [GNS][GK][NRP]
  uint64_t* full = (uint64_t*)(smem + GNS * Geo::STAGE + GNS * Geo::TF32);
  uint64_t* empty = full + GNS;
  volatile int* abort = (volatile int*)(empty + GNS);
  __shared__ float cj[CSTR];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GNS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], GemvPar<Q>::CONS);
    }
    *abort = 0;
    tc::fence_mbar_init();
  }
  for (int e = threadIdx.x; e < CSTR; e += blockDim.x) cj[e] = a.cst[e];
  __syncthreads();
  const int nkb = a.Kpad / GK;
  const int64_t snp_end = a.row0 + a.nsnp;
  const int64_t nunits = (a.nsnp + GUNIT - 1) / GUNIT;
  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_map(&mapG);
      tc::prefetch_map(&mapA);
      tc::prefetch_map(&mapT1);
      tc::prefetch_map(&mapT2);
      uint32_t h = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int row = (int)(a.row0 + u * GUNIT);
        for (int kb = 0; kb < nkb; ++kb, ++h) {
          const uint32_t s = h % GNS;
          if (h >= GNS && !tc::mbar_wait(&empty[s], ((h / GNS) - 1) & 1, a.status, abort)) { ok = false; break; }
          uint8_t* buf = smem + s * Geo::STAGE;
          const int x = kb * GK;
          tc::mbar_expect_tx(&full[s], GDATA + NR * GK * 2);
#pragma unroll
          for (int t = 0; t < 2; ++t) tc::tma_load_2d(buf + t * GBOX, &mapG, &full[s], x, row + 128 * t);
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int t = 0; t < 2; ++t)
              tc::tma_load_2d(buf + (2 + 2 * p + t) * GBOX, &mapA, &full[s], x, (int)a2_row(p, row + 128 * t));
          tc::tma_load_2d(buf + GDATA, &mapT1, &full[s], x, 0);
          tc::tma_load_2d(buf + GDATA + G1 * GK * 2, &mapT2, &full[s], x, 0);
        }
      }
      // every stage's last release must land before the CTA exits
      for (uint32_t s = 0; s < GNS && h > s; ++s) {
        const uint32_t uses = (h - s + GNS - 1) / GNS;
        tc::mbar_wait(&empty[s], (uses - 1) & 1, a.status, abort);
      }
    }
    return;
  }
  // -------------------------------------------------------------- consumers: NT SNPs per thread
  constexpr int NT = GemvPar<Q>::NT, GTHR = GemvPar<Q>::THR;
  const int ct = threadIdx.x - 32, r = ct % 128;  // row r of tiles t0 .. t0 + NT - 1
  const int t0 = NT == 2 ? 0 : ct / 128;
  const float inv_dof = 1.f / a.dof, F = 1.f / 256.f, FV = 1.f / 512.f;  // FV: the v' columns' second slice
  const int full_b = a.full_b;
  unsigned long long nsing = 0;
  uint32_t h = 0;
  bool ok = true;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    float acc[NT][G1], c2[NT][6];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
#pragma unroll
      for (int i = 0; i < G1; ++i) acc[t][i] = 0.f;
#pragma unroll
      for (int i = 0; i < 6; ++i) c2[t][i] = 0.f;
    }
    for (int kb = 0; kb < nkb; ++kb, ++h) {
      const uint32_t s = h % GNS;
      if (ok && !tc::mbar_wait(&full[s], (h / GNS) & 1, a.status, abort)) ok = false;
      const uint8_t* buf = smem + s * Geo::STAGE;
      float* tfs = tf + s * GK * NRP;
      // the stage's trait slices, bf16 [NR][GK] -> FP32 [GK][NRP]
      const __nv_bfloat16* traw = (const __nv_bfloat16*)(buf + GDATA);
      for (int idx = ct; idx < NR * GK; idx += GTHR) tfs[(idx % GK) * NRP + idx / GK] = __bfloat162float(traw[idx]);
      tc::named_sync(1, GTHR);
      const uint32_t sw = (uint32_t)((r >> 1) & 3);
#pragma unroll
      for (int c = 0; c < GK / 8; ++c) {
        const uint32_t off = (uint32_t)r * (GK * 2) + ((c ^ sw) << 4);
        float xg[NT][8], xa1[NT][8], xa2[NT][8], xa3[NT][8];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int tb = t0 + t;
          bf16x8(*(const uint4*)(buf + tb * GBOX + off), xg[t]);
          bf16x8(*(const uint4*)(buf + (2 + tb) * GBOX + off), xa1[t]);
          bf16x8(*(const uint4*)(buf + (4 + tb) * GBOX + off), xa2[t]);
          bf16x8(*(const uint4*)(buf + (6 + tb) * GBOX + off), xa3[t]);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          // the trait's row of this k: NRP floats, 8-byte aligned (NRP is even)
          const float2* tr = reinterpret_cast<const float2*>(tfs + (8 * c + e) * NRP);
          float tv[NRP];
#pragma unroll
          for (int i = 0; i < NRP / 2; ++i) {
            const float2 v2 = tr[i];
            tv[2 * i] = v2.x;
            tv[2 * i + 1] = v2.y;
          }
          const float e2s = tv[G1], e1 = tv[G1 + 1], e2 = tv[G1 + 2], e3s = tv[G1 + 3];
#pragma unroll
          for (int t = 0; t < NT; ++t) {
#pragma unroll
            for (int i = 0; i < G1; ++i) acc[t][i] = fmaf(xg[t][e], tv[i], acc[t][i]);
            c2[t][0] = fmaf(xa1[t][e], e1, c2[t][0]);   // A1 x E1   (level 0)
            c2[t][1] = fmaf(xa1[t][e], e2, c2[t][1]);   // A1 x E2
            c2[t][2] = fmaf(xa1[t][e], e3s, c2[t][2]);  // A1 x E3s
            c2[t][3] = fmaf(xa2[t][e], e2s, c2[t][3]);  // A2 x E2s
            c2[t][4] = fmaf(xa2[t][e], e1, c2[t][4]);   // A2 x E1
            c2[t][5] = fmaf(xa3[t][e], e1, c2[t][5]);   // A3s x E1
          }
        }
      }
      // release the stage: one arrival per warp once all its lanes have read it
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&empty[s]);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int64_t snp = a.row0 + u * GUNIT + 128 * (t0 + t) + r;
      const bool valid = ok && snp >= a.snp_lo && snp < snp_end;
      if (!valid) continue;
      const float* acc_t = acc[t];
      const float* c2t = c2[t];
      // the fused kernel's epilogue for pair (snp, trait 0)
      const float sA = a.sA[snp];
      const float num =
          cj[0] * fmaf(F, fmaf(F, fmaf(F, acc_t[3 + 2 * PM1], acc_t[2 + 2 * PM1]), acc_t[1 + PM1]), acc_t[0]);
      float z[Q1], zz = 0.f;
#pragma unroll
      for (int c = 0; c < PM1; ++c) {
        z[c] = cj[1 + c] * fmaf(FV, acc_t[2 + PM1 + c], acc_t[1 + c]);
        zz = fmaf(z[c], z[c], zz);
      }
      const float lvl1 = (c2t[1] + c2t[2]) + (c2t[3] + c2t[4]) + c2t[5];
      const float sv = (sA * cj[cst_escale(Q)]) * fmaf(F, lvl1, c2t[0]);
      const float delta = sv - zz;
      float beta, se;
      const bool sing = !(delta > 1e-6f * sv) || !(sA > 0.f);
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
  }
  for (int o = 16; o > 0; o >>= 1) nsing += __shfl_xor_sync(0xffffffffu, nsing, o);
  if (lane == 0 && nsing) atomicAdd(a.singular, nsing);
}


// Launches gemv1_kernel<Q> (maps built by the caller).
template <int Q>
int launch_gemv1_q(gwas_ctx* c, const FusedArgs& a, const CUtensorMap& mg, const CUtensorMap& ma, const CUtensorMap& m1,
                   const CUtensorMap& m2) {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t units = (a.nsnp + GUNIT - 1) / GUNIT;
  const unsigned blocks = (unsigned)std::min<int64_t>(nsm, units);
  auto kern = gemv1_kernel<Q>;
  constexpr int smem = GemvGeo<Q>::SMEM;
  static_assert(smem <= 227 * 1024, "single-trait kernel shared memory");
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  ProfScope ps(c, "gemv1");
  kern<<<blocks, 32 + GemvPar<Q>::THR, smem, c->stream>>>(mg, ma, m1, m2, a);
  c->launches++;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(c, GWAS_ERR_CUDA, std::string("single-trait kernel launch: ") + cudaGetErrorString(e));
  return GWAS_OK;
}

}  // namespace
