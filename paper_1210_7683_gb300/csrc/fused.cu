// Fused contraction + per-pair Schur-complement solve on the tensor cores (the loop
// body of Algorithm 5: S_BL, S_BR, b_B for every SNP x trait pair, then the p x p
// solve, with the blocks of Algorithm 2).
//
// Per pair (i, j), with x_c = P_c x_i the SNP centred against span(X_L) (an exact
// reparametrisation: the SNP coefficient and its standard error do not change, the
// covariate coefficients move by a_i * beta), r_j the GLS residual of y_j on X_L,
// L_j the Cholesky factor of S_TL,j and e_j = diag(D_j^-1):
//   num  = x_i^T M_j^-1 r_j                  = x_i . w_j       (C1, column w)
//   z    = L_j^-1 X_L^T M_j^-1 x_c           = x_i . v'_j,c    (C1, columns v)
//   s    = x_c^T M_j^-1 x_c = sum_k e_jk x'_ck^2                (C2)
//   delta = s - z^T z  (Schur complement of S_TL in S),  beta = num / delta,
//   RSS = r_j^T M_j^-1 r_j - num * beta,  SE = sqrt(RSS / ((n - p) delta)).
// C1 contracts the exact int8 genotypes (as bf16) against fixed-point slices of
// the per-trait columns [w | v'_1..3]; C2 contracts slices of x'_c^2 against slices
// of e_j.  Level-0 slice products are exact in FP32 (bounded partial sums), the
// lower levels go to separate accumulators, and the levels are recombined in the
// epilogue.
//
// Tile: 128 SNPs (TMEM lanes) x 32 traits.  TMEM columns:
//   [0,128)   C1 level 0  (slice 1 of w, v1, v2, v3; 32 traits each)
//   [128,256) C1 level 1  (slice 2)
//   [256,288) w slice 3   [288,320) w slice 4
//   [320,352) C2 level 0  [352,384) C2 level-1 units (a)  [384,416) (b)
#include <algorithm>
#include <cstdio>

#include "fused.cuh"
#include "gwas_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int BM = 128, TT = 32, BK = 64;
constexpr int PM1 = 3;
constexpr int G_BYTES = BM * BK * 2;                 // 16 KB: one A tile
constexpr int B1_ROWS = 10 * TT, B2_ROWS = 4 * TT;   // 320 and 128 rows
constexpr int SLOT = 64 * 1024;                      // a ring slot holds either half-stage
constexpr int SLOTS = 3;
constexpr int H1_BYTES = G_BYTES + B1_ROWS * BK * 2; // 57344
constexpr int H2_BYTES = 3 * G_BYTES + B2_ROWS * BK * 2;  // 65536
constexpr int SMEM_BYTES = SLOTS * SLOT + 1024 + 512;
constexpr int TMEM_COLS = 512;
static_assert(H1_BYTES <= SLOT && H2_BYTES <= SLOT, "half-stage does not fit a slot");

__device__ __forceinline__ void tile_coords(int tile, const FusedArgs& a, int& st, int& tt) {
  const int per_group = a.group * a.n_ttiles;
  const int g = tile / per_group;
  const int w = tile % per_group;
  const int g0 = g * a.group;
  const int gs = min(a.group, a.n_stiles - g0);
  tt = w / gs;
  st = g0 + w % gs;
}

__global__ void __launch_bounds__(192, 1) fused_kernel(const __grid_constant__ CUtensorMap mapG,
                                                       const __grid_constant__ CUtensorMap mapA2,
                                                       const __grid_constant__ CUtensorMap mapB1,
                                                       const __grid_constant__ CUtensorMap mapB2, FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + SLOTS * SLOT);
  uint64_t* empty = full + SLOTS;
  uint64_t* acc_full = empty + SLOTS;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tslot = (uint32_t*)(acc_empty + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ntiles = a.n_stiles * a.n_ttiles;
  const int nkb = a.Kpad / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, 4);
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tslot, TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_map(&mapG);
      tc::prefetch_map(&mapA2);
      tc::prefetch_map(&mapB1);
      tc::prefetch_map(&mapB2);
      uint32_t h = 0;  // half-stage counter
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int st, tt;
        tile_coords(tile, a, st, tt);
        const int row = a.row0 + st * BM;
        for (int kb = 0; kb < nkb && ok; ++kb) {
          for (int half = 0; half < 2; ++half, ++h) {
            const uint32_t s = h % SLOTS;
            if (h >= SLOTS && !tc::mbar_wait(&empty[s], ((h / SLOTS) - 1) & 1, a.status, abort)) { ok = false; break; }
            uint8_t* buf = smem + s * SLOT;
            const int x = kb * BK;
            if (half == 0) {
              tc::mbar_expect_tx(&full[s], H1_BYTES);
              tc::tma_load_2d(buf, &mapG, &full[s], x, row);
#pragma unroll
              for (int q = 0; q < B1_ROWS / 64; ++q)
                tc::tma_load_2d(buf + G_BYTES + q * 64 * BK * 2, &mapB1, &full[s], x, tt * B1_ROWS + q * 64);
            } else {
              tc::mbar_expect_tx(&full[s], H2_BYTES);
#pragma unroll
              for (int p = 0; p < 3; ++p) tc::tma_load_2d(buf + p * G_BYTES, &mapA2, &full[s], x, p * a.mpad + row);
#pragma unroll
              for (int q = 0; q < B2_ROWS / 64; ++q)
                tc::tma_load_2d(buf + 3 * G_BYTES + q * 64 * BK * 2, &mapB2, &full[s], x, tt * B2_ROWS + q * 64);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t id256 = tc::idesc_bf16(BM, 8 * TT), id64 = tc::idesc_bf16(BM, 2 * TT);
      constexpr uint32_t id96 = tc::idesc_bf16(BM, 3 * TT), id32 = tc::idesc_bf16(BM, TT);
      uint32_t h = 0, tcount = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tcount) {
        if (tcount > 0 && !tc::mbar_wait(acc_empty, (tcount - 1) & 1, a.status, abort)) { ok = false; break; }
        tc::fence_after();
        for (int kb = 0; kb < nkb && ok; ++kb) {
          for (int half = 0; half < 2; ++half, ++h) {
            const uint32_t s = h % SLOTS;
            if (!tc::mbar_wait(&full[s], (h / SLOTS) & 1, a.status, abort)) { ok = false; break; }
            tc::fence_after();
            uint8_t* buf = smem + s * SLOT;
            if (half == 0) {
              const uint64_t dg = tc::sdesc_sw128(buf);
              const uint64_t db = tc::sdesc_sw128(buf + G_BYTES);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint32_t acc = (kb | k) ? 1u : 0u;
                tc::mma_bf16(tbase + 0, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, k * 32), id256, acc);
                tc::mma_bf16(tbase + 8 * TT, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, 8 * TT * 128 + k * 32),
                             id64, acc);
              }
            } else {
              const uint64_t d1 = tc::sdesc_sw128(buf), d2 = tc::sdesc_sw128(buf + G_BYTES);
              const uint64_t d3 = tc::sdesc_sw128(buf + 2 * G_BYTES), de = tc::sdesc_sw128(buf + 3 * G_BYTES);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint32_t acc = (kb | k) ? 1u : 0u;
                // A1 x [E1 | E2 | E3s] -> [level 0 | a | b]
                tc::mma_bf16(tbase + 10 * TT, tc::sdesc_add(d1, k * 32), tc::sdesc_add(de, TT * 128 + k * 32), id96, acc);
                // A2 x [E2s | E1] -> [a | b]
                tc::mma_bf16(tbase + 11 * TT, tc::sdesc_add(d2, k * 32), tc::sdesc_add(de, k * 32), id64, 1u);
                // A3s x E1 -> a
                tc::mma_bf16(tbase + 11 * TT, tc::sdesc_add(d3, k * 32), tc::sdesc_add(de, TT * 128 + k * 32), id32, 1u);
              }
            }
            tc::mma_commit(&empty[s]);
          }
        }
        if (ok) tc::mma_commit(acc_full);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp % 4;                    // TMEM lane quarter
    const uint32_t lane_base = tbase + ((uint32_t)(q * 32) << 16);
    uint32_t tcount = 0;
    unsigned long long nsing = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tcount) {
      int st, tt;
      tile_coords(tile, a, st, tt);
      const bool ok = tc::mbar_wait(acc_full, tcount & 1, a.status, abort);
      tc::fence_after();
      const int64_t i = (int64_t)st * BM + q * 32 + lane;   // SNP index relative to row0
      const bool valid_i = ok && i < a.nsnp;
      const float sA = valid_i ? a.sA[a.row0 + i] : 0.f;
      float ac[PM1] = {0.f, 0.f, 0.f};
      if (valid_i && a.full_b) {
#pragma unroll
        for (int c = 0; c < PM1; ++c) ac[c] = a.acoef[(a.row0 + i) * PM1 + c];
      }
      for (int j0 = 0; j0 < TT; j0 += 8) {
        uint32_t hw[8], hz[3][8], lw[8], lz[3][8], w3[8], w4[8], d0[8], da[8], db[8];
        tc::tmem_ld8(lane_base + 0 * TT + j0, hw);
#pragma unroll
        for (int c = 0; c < PM1; ++c) tc::tmem_ld8(lane_base + (1 + c) * TT + j0, hz[c]);
        tc::tmem_ld8(lane_base + 4 * TT + j0, lw);
#pragma unroll
        for (int c = 0; c < PM1; ++c) tc::tmem_ld8(lane_base + (5 + c) * TT + j0, lz[c]);
        tc::tmem_ld8(lane_base + 8 * TT + j0, w3);
        tc::tmem_ld8(lane_base + 9 * TT + j0, w4);
        tc::tmem_ld8(lane_base + 10 * TT + j0, d0);
        tc::tmem_ld8(lane_base + 11 * TT + j0, da);
        tc::tmem_ld8(lane_base + 12 * TT + j0, db);
        tc::tmem_ld_wait();
        tc::reg_fence(hw); tc::reg_fence(lw); tc::reg_fence(w3); tc::reg_fence(w4);
        tc::reg_fence(d0); tc::reg_fence(da); tc::reg_fence(db);
#pragma unroll
        for (int c = 0; c < PM1; ++c) { tc::reg_fence(hz[c]); tc::reg_fence(lz[c]); }
        if (j0 + 8 == TT) {
          // every TMEM read of this tile is complete: release the accumulators
          tc::fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(acc_empty);
        }
        if (!valid_i) continue;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int jj = tt * TT + j0 + u;     // trait index within the block
          if (jj >= a.ntrait) break;
          const float* cj = a.cst + (size_t)jj * FUSED_CST;
          const float F = 1.f / 256.f;
          const float num = cj[0] * fmaf(F, fmaf(F, fmaf(F, __uint_as_float(w4[u]), __uint_as_float(w3[u])),
                                                 __uint_as_float(lw[u])), __uint_as_float(hw[u]));
          float z[PM1], zz = 0.f;
#pragma unroll
          for (int c = 0; c < PM1; ++c) {
            z[c] = cj[1 + c] * fmaf(F, __uint_as_float(lz[c][u]), __uint_as_float(hz[c][u]));
            zz = fmaf(z[c], z[c], zz);
          }
          const float s = (sA * cj[4]) * fmaf(F, __uint_as_float(da[u]) + __uint_as_float(db[u]), __uint_as_float(d0[u]));
          const float delta = s - zz;
          float beta, se;
          const bool sing = !(delta > 1e-6f * s) || !(sA > 0.f);
          if (sing) {
            beta = se = __int_as_float(0x7fc00000);
            ++nsing;
          } else {
            beta = num / delta;
            const float rss = fmaxf(fmaf(-num, beta, cj[5]), 0.f);
            se = sqrtf(rss / (a.dof * delta));
          }
          const int64_t o = (int64_t)jj * a.ldo + (a.row0 + i - a.i0);
          if (a.full_b) {
            double* ob = a.out_b64 + o * (PM1 + 1);
#pragma unroll
            for (int c = 0; c < PM1; ++c) {
              // beta_L = g - L^-T z beta - a_i beta
              float t = cj[6 + c];
#pragma unroll
              for (int d = 0; d < PM1; ++d) t = fmaf(-cj[9 + c * PM1 + d] * z[d], beta, t);
              t = fmaf(-ac[c], beta, t);
              ob[c] = sing ? (double)beta : (double)t;
            }
            ob[PM1] = (double)beta;
          } else {
            a.out_beta[o] = beta;
            a.out_se[o] = se;
          }
        }
      }
    }
    // warp-aggregated count of singular pairs
    for (int o = 16; o > 0; o >>= 1) nsing += __shfl_xor_sync(0xffffffffu, nsing, o);
    if (lane == 0 && nsing) atomicAdd(a.singular, nsing);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace

int launch_fused(gwas_ctx* c, const FusedArgs& args, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2) {
  CUtensorMap mg, ma, m1, m2;
  FusedArgs a = args;
  if (!make_bf16_map(&mg, G, a.mpad, a.Kpad, BM) || !make_bf16_map(&ma, A2, 3ull * a.mpad, a.Kpad, BM) ||
      !make_bf16_map(&m1, B1, (uint64_t)a.n_ttiles * B1_ROWS, a.Kpad, 64) ||
      !make_bf16_map(&m2, B2, (uint64_t)a.n_ttiles * B2_ROWS, a.Kpad, 64))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  static int nsm = 0;
  if (!nsm) {
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    cudaFuncSetAttribute(fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  }
  const int ntiles = a.n_stiles * a.n_ttiles;
  if (ntiles == 0) return GWAS_OK;
  const int grid = std::min(ntiles, a.max_ctas > 0 ? a.max_ctas : nsm);
  ProfScope ps(c, "fused");
  fused_kernel<<<grid, 192, SMEM_BYTES, c->stream>>>(mg, ma, m1, m2, a);
  c->launches++;
  return GWAS_OK;
}
