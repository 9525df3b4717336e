#pragma once
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
// Work is split into tiles of 128 SNPs x TT traits (TT = 32 for p = 4), one CTA per tile,
// or (the optional CTA-pair shape, p = 4) a pair of CTAs on two SNP tiles and one trait
// tile issuing M = 256 MMAs (cta_group::2), each CTA loading its own SNP rows and half of
// the trait rows.
// TMEM columns of each CTA for p = 4:
//   [0,128)   C1 level 0  (slice 1 of w, v1, v2, v3; 32 traits each)
//   [128,256) C1 level 1  (slice 2)
//   [256,288) w slice 3   [288,320) w slice 4
//   [320,416) A1 x [E1 | E2 | E3s]: C2 level 0, then two groups in level-1 units
//   [416,480) A2 x [E2s | E1]       [480,512) A3s x E1   (level-1 units)
// Other p keep the order with (1 + q) groups per C1 level (q = p - 1) and TT = 16 traits
// for q <= 10, TT = 8 above (fused.cuh); 8-trait tiles widen A1 to [E2s | E1 | E2 | E3s]
// and A3s to [E1 | E2] (M = 128 MMAs need N % 16 == 0), leaving two groups unused.
// Every MMA of a K step writes its own columns, so consecutive small MMAs do not wait
// on one another's accumulator (a chain of dependent N <= 128 MMAs runs at the MMA
// latency, not at the tensor-core rate); the epilogue adds the level-1 groups.
// With S_BR interpolated (INTERP, the default where its bound holds) the C2 columns are
// not used and the K loop streams only the C1 operands; at p = 4 its tiles hold 24 traits
// (C1 = 240 columns, one MMA per K step), accumulated alternately in [0, 240) and [256, 496)
// so that a tile's MMAs overlap the epilogue of the one before.  The CTA pair of that kernel
// can contract e2m1 operands instead of bf16 (FP4, see fused_kernel): its constant scale
// factors sit in [240, 256) and [496, 512), and a 15th warp stages the epilogue's per-tile data.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "fused.cuh"
#include "gwas_internal.cuh"
#include "tc.cuh"

namespace {

// K extent of one stage: 64 bf16 = one 128-byte swizzled row.  (32-wide stages with
// the 64-byte swizzle and 32-row boxes measured 1.6x slower: the TMA unit's cost per box.)
constexpr int BM = 128, BK = 64;
constexpr int ROWB = BK * 2;                         // bytes per operand row of a stage
constexpr int G_BYTES = BM * ROWB;                   // 16 KB: one A tile
constexpr int SLOT = 64 * 1024;                      // one-CTA shapes: a ring slot holds either half-stage
constexpr int SLOTS = 3;
// half-stages of the one-CTA shapes: G + the C1 trait rows; the three x'^2 planes + the C2 trait rows
__host__ __device__ constexpr int h1_bytes(int q) { return G_BYTES + c1_rows(q) * ROWB; }
__host__ __device__ constexpr int h2_bytes(int q) { return 3 * G_BYTES + c2_rows(q) * ROWB; }
// CTA pair (q = 3): each CTA stages its own SNP rows and half of the trait rows, in three items
// per K block (G + C1 half: 36 KB; C2 half + A1: 28 KB; A2 + A3s: 32 KB) and a ring of six
// 36 KB slots, i.e. two K blocks in flight.
constexpr int PSLOT = 36 * 1024, PSLOTS = 6;
// With S_BR interpolated a K block is one item: the genotype tile and the C1 trait rows (one CTA),
// or the CTA's own genotype rows and its half of the C1 rows (pair).  At q = 3 the 24-trait tiles
// make that 46 KB (one CTA, 4 slots) or 31 KB (pair, 6 slots).
__host__ __device__ constexpr int interp_item_bytes(int q, bool pair) {
  return G_BYTES + (pair ? c1_rows_of(q, true) / 2 : c1_rows_of(q, true)) * ROWB;
}
__host__ __device__ constexpr int interp_slots(int q, bool pair) { return pair ? 6 : q == 3 ? 4 : 3; }
constexpr int PC1_ROWS = c1_rows(3) / 2, PC2_ROWS = c2_alloc(3) / 2;  // 160 and 96 trait rows per CTA
constexpr int PI0_BYTES = G_BYTES + PC1_ROWS * ROWB;   // G + this CTA's C1 trait rows
constexpr int PI1_BYTES = PC2_ROWS * ROWB + G_BYTES;   // this CTA's C2 trait rows + A1
constexpr int PI2_BYTES = 2 * G_BYTES;                 // A2 + A3s
__host__ __device__ constexpr int cst_bytes(int q) { return mixed_tt(q) * cst_stride(q) * 4; }  // one tile's constants
__host__ __device__ constexpr int slot_bytes(bool interp, int q, bool pair = false) {
  return interp ? (interp_item_bytes(q, pair) + 1023) / 1024 * 1024 : pair ? PSLOT : SLOT;
}
__host__ __device__ constexpr int ring_bytes(bool pair, bool interp, int q) {
  return (interp ? interp_slots(q, pair) : pair ? PSLOTS : SLOTS) * slot_bytes(interp, q, pair);
}
// INTERP: the tile's Chebyshev coefficients [CHEB_MAX_R + 1][128 SNPs] and T_k(x_j) [CHEB_MAX_R][TT].
// The CTA pair stages them one tile ahead by bulk copies: two buffers of the coefficients and of T
// as stored ([TT][CHEB_MAX_R]), and one array of T transposed for the series.
__host__ __device__ constexpr int cheb_pair_buf(int q) { return (CHEB_MAX_R + 1) * 128 + tile_traits(q, true) * CHEB_MAX_R; }
__host__ __device__ constexpr int cheb_stage_bytes(bool interp, int q, bool pair = false) {
  return !interp ? 0
         : pair  ? (2 * cheb_pair_buf(q) + CHEB_MAX_R * tile_traits(q, true)) * 4
                 : ((CHEB_MAX_R + 1) * 128 + CHEB_MAX_R * mixed_tt(q)) * 4;
}
__host__ __device__ constexpr int smem_bytes(bool pair, int q, bool interp = false) {
  return ring_bytes(pair, interp, q) + 2 * cst_bytes(q) + cheb_stage_bytes(interp, q, pair) + 1024 + 512;
}
// e2m1 operands (the interpolated CTA pair, q = 3): a ring item is one K block of 256, i.e. one
// 128-byte row of packed e2m1 values per operand row: the CTA's 128 genotype rows and its 120 C1
// rows in each of the three digits (16 KB + 45 KB), in three slots.
constexpr int BK4 = 256;
constexpr int F4_HALF = 120;
constexpr int F4_ITEM = G_BYTES + 3 * F4_HALF * ROWB;
constexpr int F4_SLOTS = 3;
// TMEM columns of the constant scale factors, beside the accumulator buffers [0, 240) and [256, 496)
constexpr int SF_A = 240, SF_B0 = 248, SF_B1 = 496, SF_B2 = 504;
__host__ __device__ constexpr int smem_bytes_fp4() {
  return F4_SLOTS * F4_ITEM + 2 * cst_bytes(3) + cheb_stage_bytes(true, 3, true) + 1024 + 512;
}
static_assert(F4_ITEM % 1024 == 0 && (F4_HALF * ROWB) % 1024 == 0 && smem_bytes_fp4() <= 227 * 1024, "e2m1 ring");
static_assert(2 * F4_HALF == c1_rows_of(3, true), "e2m1 C1 rows");
constexpr int TMEM_COLS = 512;
constexpr bool fits_all_q() {
  for (int q = 0; q <= MIXED_MAX_Q; ++q)
    if (h1_bytes(q) > SLOT || h2_bytes(q) > SLOT || smem_bytes(false, q) > 227 * 1024 ||
        smem_bytes(false, q, true) > 227 * 1024 || c1_rows_of(q, true) > 512)
      return false;
  return true;
}
static_assert(fits_all_q(), "half-stage does not fit a slot");
static_assert(PI0_BYTES <= PSLOT && PI1_BYTES <= PSLOT && PI2_BYTES <= PSLOT, "pair item does not fit a slot");
static_assert(smem_bytes(true, 3) <= 227 * 1024 && smem_bytes(true, 3, true) <= 227 * 1024, "shared memory");

// epilogue warps EPW for TT traits per tile: four lane quarters, each warp owning TT / (EPW / 4)
// traits, read from TMEM in groups of 4
__host__ __device__ constexpr bool JPW_OK(int tt, int epw) { return epw % 4 == 0 && tt % (epw / 4) == 0 && (tt / (epw / 4)) % 4 == 0; }
// the epilogue warps of the interpolated kernel: 12 for its 24-trait tiles (8 traits per warp)
__host__ __device__ constexpr int epw_interp(int q) { return tile_traits(q, true) == 24 ? 12 : mixed_tt(q) == 8 ? 8 : 16; }
// the epilogue warps of a tile width: 16, or 8 for 8-trait tiles
__host__ __device__ constexpr int epw_for(int q) { return mixed_tt(q) == 8 ? 8 : 16; }

template <int CS>
__device__ __forceinline__ void super_coords(int u, const FusedArgs& a, int& us, int& ut) {
  const int nss = (a.n_stiles + CS - 1) / CS, nst = a.n_ttiles;
  const int per_group = a.group * nst;
  const int g = u / per_group;
  const int w = u % per_group;
  const int g0 = g * a.group;
  const int gs = min(a.group, nss - g0);
  ut = w / gs;
  us = g0 + w % gs;
}

// Q = p - 1 covariates.  PAIR: the two CTAs of a cluster issue one M = 256 MMA
// (cta_group::2); each holds its own 128 SNP rows and half of every MMA's trait rows (the
// pair layout of the C2 operand, c2_alloc rows per tile), the leader (rank 0) issues the
// MMAs, and both CTAs' loads complete on the leader's barriers.
// INTERP: S_BR is not contracted here but evaluated per pair from its Chebyshev series in
// h^2 (FusedArgs::cheb_*): the K loop streams only the C1 operands (genotypes and the trait
// columns [w | v']), one item per K block.
// FP4 (PAIR, INTERP, q = 3): the C1 operands as e2m1 values (kind::mxf4).  A fixed-point slice
// digit q (|q| <= 256; the split covers -288..287) is 64 d0 + 8 d1 + d2, d in [-4, 4], and the three digits are
// contracted into the slice's own accumulator by MMAs whose B scale factors are 2^6, 2^3 and 2^0:
// every partial sum is the same integer as the bf16 kernel's, so the outputs do not change.
// Threads of a CTA: the TMA producer and MMA warps, EPW epilogue warps and, in the interpolated
// CTA pair, a warp that stages the epilogue's per-tile data.
__host__ __device__ constexpr int fused_threads(int epw, bool pair, bool interp) { return 64 + 32 * epw + (pair && interp ? 32 : 0); }

template <int EPW, bool SERVE, bool PAIR, int Q, bool INTERP = false, bool FP4 = false>
__global__ void __launch_bounds__(fused_threads(EPW, PAIR, INTERP), 1)
    fused_kernel(const __grid_constant__ CUtensorMap mapG, const __grid_constant__ CUtensorMap mapA2,
                 const __grid_constant__ CUtensorMap mapB1, const __grid_constant__ CUtensorMap mapB2, FusedArgs a) {
  constexpr int CS = PAIR ? 2 : 1;                  // SNP tiles per cluster (the CTA pair: 2)
  static_assert(!PAIR || (!SERVE && Q == 3), "the pair shape is built for q = 3 outside serving");
  static_assert(!INTERP || !SERVE, "the interpolated S_BR is built for the solve kernels");
  static_assert(!FP4 || (PAIR && INTERP && Q == 3), "the e2m1 operands are built for the interpolated pair");
  constexpr int PM1 = Q, Q1 = Q > 0 ? Q : 1, TT = tile_traits(Q, INTERP), CSTR = cst_stride(Q);
  constexpr int B1_ROWS = c1_groups(Q) * TT, B2_ROWS = c2_rows(Q), B2_ROWS_PAIR = c2_alloc(Q);
  // the pair with S_BR interpolated: one MMA of N = B1_ROWS per K step, each CTA holding half of its rows
  constexpr int PC1I = B1_ROWS / 2, PI0I = G_BYTES + PC1I * ROWB;
  static_assert(!(PAIR && INTERP) || B1_ROWS <= 256, "the interpolated pair issues one MMA per K step");
  constexpr int C2B = c1_groups(Q) * TT;            // first TMEM column of the C2 accumulators
  // 8-trait tiles widen two C2 MMAs to N = 16 multiples: A1 also multiplies E2s (one unused
  // group in front), A3s also E2 (one unused group at the end)
  constexpr int C2_OFF = TT == 8 ? TT : 0;
  static_assert(JPW_OK(TT, EPW), "epilogue warps: each must own a multiple of 4 traits");
  constexpr int H1_BYTES = G_BYTES + B1_ROWS * ROWB, H2_BYTES = h2_bytes(Q);
  // C1 MMAs of the one-CTA shapes: the C1 trait rows in chunks of at most 256 (N <= 256)
  constexpr int N0 = B1_ROWS < 256 ? B1_ROWS : 256, N1 = B1_ROWS - N0;
  // TMA boxes of the C1 trait rows in the one-CTA shapes (at most 256 rows per box)
  constexpr int B1_NBOX = B1_ROWS <= 256 ? 1 : 2, B1_BOX = B1_ROWS / B1_NBOX;
  static_assert(N1 >= 0 && N1 <= 256 && N0 % 16 == 0 && N1 % 16 == 0 && B1_BOX % 8 == 0, "C1 geometry");
  // One CTA per tile: every half-stage is three TMA boxes of 128 to 192 rows (the genotype
  // tile and the C1 trait rows in one or two boxes; the three x'^2 planes, stored next to
  // one another, in two halves and the C2 trait rows).  The TMA unit pays a fixed cost per
  // box of the order of 50 cycles, so large boxes keep the load rate up.
  constexpr int NSL = FP4 ? F4_SLOTS : INTERP ? interp_slots(Q, PAIR) : PAIR ? PSLOTS : SLOTS;  // ring slots
  constexpr int SLB = FP4 ? F4_ITEM : slot_bytes(INTERP, Q, PAIR);                             // and their size
  constexpr int NI = INTERP ? 1 : PAIR ? 3 : 2;                           // ring items per K block
  constexpr int RING = FP4 ? F4_SLOTS * F4_ITEM : ring_bytes(PAIR, INTERP, Q);
  // Double-buffered accumulators where a tile's C1 columns fit 256 (with S_BR interpolated: at
  // p = 4 the 24-trait tiles): tile u accumulates into columns [256 (u & 1), +B1_ROWS), so the
  // MMAs of the next tile do not wait for the epilogue to read this one.
  constexpr bool DB = INTERP && B1_ROWS <= 256;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // PSTAGE (the interpolated CTA pair): a tile's constants, Chebyshev coefficients and T_k(x_j) are
  // copied by one thread with bulk copies while the tile before is in the epilogue
  constexpr bool PSTAGE = PAIR && INTERP;
  constexpr int CBUF = cheb_pair_buf(Q);
  float* cst_smem = (float*)(smem + RING);  // [2][TT][CSTR], double-buffered by tile
  float* cheb_c = (float*)(smem + RING + 2 * cst_bytes(Q));  // INTERP: [CHEB_MAX_R + 1][128]
  float* cheb_t = cheb_c + (CHEB_MAX_R + 1) * 128;          // INTERP, one CTA: [CHEB_MAX_R][TT]
  // PSTAGE: buffers b = 0, 1 at cheb_c + b * CBUF (coefficients [CHEB_MAX_R + 1][128], then T as
  // [TT][CHEB_MAX_R]) and T transposed, [CHEB_MAX_R][TT], at cheb_c + 2 * CBUF
  uint64_t* full = (uint64_t*)(smem + RING + 2 * cst_bytes(Q) + cheb_stage_bytes(INTERP, Q, PAIR));
  uint64_t* empty = full + NSL;
  uint64_t* acc_full = empty + NSL;          // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* stage_full = acc_empty + 2;      // [2] PSTAGE
  uint64_t* stage_empty = stage_full + 2;    // [2] PSTAGE
  uint32_t* tslot = (uint32_t*)(stage_empty + 2);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t crank = 0, cid = blockIdx.x, ncl = gridDim.x;
  if (PAIR) {
    crank = tc::cluster_ctarank();
    cid = tc::cluster_id_x();
    ncl = tc::cluster_count_x();
  }
  const int sr = (int)crank;       // this CTA's SNP tile within the cluster
  // serving: the round's work units (from device memory when the launch is a captured graph's)
  const int nsuper = SERVE ? (a.nunits_dev ? min(*a.nunits_dev, a.nunits) : a.nunits)
                           : ((a.n_stiles + CS - 1) / CS) * a.n_ttiles;
  const int nkb = FP4 ? a.Kp4 / BK4 : a.Kpad / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSL; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], PAIR ? 2 * EPW : EPW);
      tc::mbar_init(&stage_full[b], 1);
      tc::mbar_init(&stage_empty[b], EPW);
    }
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    if (PAIR) tc::tmem_alloc_pair(tslot, TMEM_COLS);
    else tc::tmem_alloc(tslot, TMEM_COLS);
  }
  tc::fence_before();
  __syncthreads();
  if (PAIR) tc::cluster_sync();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const bool leader = !PAIR || crank == 0;
  if (FP4) {
    // the scale factors: 1 for the genotypes, 2^6, 2^3, 2^0 for the three digits of the trait
    // columns (UE8M0 bytes), in every lane of both CTAs before the first MMA
    if (warp >= 2 && warp < 6) {
      const uint32_t lanes = tbase + ((uint32_t)((warp % 4) * 32) << 16);
      tc::tmem_st8_fill(lanes + SF_A, 0x7F7F7F7Fu);
      tc::tmem_st8_fill(lanes + SF_B0, 0x85858585u);
      tc::tmem_st8_fill(lanes + SF_B1, 0x82828282u);
      tc::tmem_st8_fill(lanes + SF_B2, 0x7F7F7F7Fu);
      tc::tmem_st_wait();
    }
    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();
    tc::fence_after();
  }

  // PSTAGE: the copies of tile uu's constants (TT traits; all allocated), its SNPs' Chebyshev
  // coefficient rows 0..CHEB_MAX_R (one TMA box from mapA2, which the interpolated kernels do not
  // otherwise use; the pair's tile past the last SNP tile reads the fill value and stores nothing)
  // and its traits' T_k(x_j) (only those of the block) into buffer b
  auto issue_stage = [&](int uu, int b) {
    int us, ut;
    super_coords<CS>(uu, a, us, ut);
    const int64_t s0 = a.row0 + (int64_t)(us * CS + sr) * BM;
    const int jb = ut * TT, nvt = min(TT, a.ntrait - jb);
    float* cc = cheb_c + b * CBUF;
    tc::mbar_expect_tx(&stage_full[b], TT * CSTR * 4 + (CHEB_MAX_R + 1) * 128 * 4 + nvt * CHEB_MAX_R * 4);
    tc::bulk_copy_g2s(cst_smem + b * TT * CSTR, a.cst + (size_t)jb * CSTR, TT * CSTR * 4, &stage_full[b]);
    tc::tma_load_2d(cc, &mapA2, &stage_full[b], (int)s0, 0);
    tc::bulk_copy_g2s(cc + (CHEB_MAX_R + 1) * 128, a.cheb_T + (size_t)jb * CHEB_MAX_R, nvt * CHEB_MAX_R * 4,
                      &stage_full[b]);
  };
  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_map(&mapG);
      tc::prefetch_map(&mapA2);
      tc::prefetch_map(&mapB1);
      tc::prefetch_map(&mapB2);
      uint32_t h = 0;  // ring item counter
      bool ok = true;
      for (int u = cid; u < nsuper && ok; u += ncl) {
        int row, tt;
        if (SERVE) {
          const int4 w = a.units[u];
          row = w.x;
          tt = w.y;
        } else {
          int us, ut;
          super_coords<CS>(u, a, us, ut);
          row = (int)a.row0 + (us * CS + sr) * BM;
          tt = ut;
          if (!PAIR && u + (int)ncl < nsuper) {
            // When the next unit starts a new trait tile, its first two K blocks of trait
            // operands are prefetched into L2: the 16 CTAs of a traversal group start that tile
            // together and would otherwise all wait on its first DRAM reads.  Measured at
            // p = 4, n = 1000: 285.6 -> 281.7 ms; prefetching 3, 4, 8 or 16 blocks was slower.
            int us2, ut2;
            super_coords<CS>(u + ncl, a, us2, ut2);
            if (ut2 != ut) {
              constexpr int PREFETCH_KB = 2;
              const int kbe = PREFETCH_KB < nkb ? PREFETCH_KB : nkb;
              for (int kb = 0; kb < kbe; ++kb) {
                for (int b = 0; b < B1_NBOX; ++b) tc::tma_prefetch_2d(&mapB1, kb * BK, ut2 * B1_ROWS + b * B1_BOX);
                if (!INTERP) tc::tma_prefetch_2d(&mapB2, kb * BK, ut2 * B2_ROWS);
              }
            }
          }
        }
        for (int kb = 0; kb < nkb && ok; ++kb) {
          for (int it = 0; it < NI; ++it, ++h) {
            const uint32_t s = h % NSL;
            if (h >= NSL && !tc::mbar_wait(&empty[s], ((h / NSL) - 1) & 1, a.status, abort)) { ok = false; break; }
            uint8_t* buf = smem + s * SLB;
            const int x = kb * BK;
            const int half = it;
            if (PAIR) {
              // own SNP rows and own half of the trait rows, completing on the leader's barrier
              const uint32_t fb = tc::mapa(&full[s], 0);
              if (FP4) {
                // the K block's 128 bytes of each of the CTA's genotype rows and of its C1 rows
                // of each digit
                if (leader) tc::mbar_expect_tx(&full[s], 2 * F4_ITEM);
                const int xb = kb * ROWB;
                tc::tma_load_2d_pair(buf, &mapG, fb, xb, row);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                  tc::tma_load_2d_pair(buf + G_BYTES + d * F4_HALF * ROWB, &mapB1, fb, xb,
                                       ((tt * 2 + (int)crank) * 3 + d) * F4_HALF);
                continue;
              }
              if (leader)
                tc::mbar_expect_tx(&full[s], 2 * (INTERP ? PI0I : it == 0 ? PI0_BYTES : it == 1 ? PI1_BYTES : PI2_BYTES));
              if (it == 0) {
                tc::tma_load_2d_pair(buf, &mapG, fb, x, row);
                tc::tma_load_2d_pair(buf + G_BYTES, &mapB1, fb, x,
                                     tt * B1_ROWS + (int)crank * (INTERP ? PC1I : PC1_ROWS));
              } else if (it == 1) {
                tc::tma_load_2d_pair(buf, &mapB2, fb, x, tt * B2_ROWS_PAIR + (int)crank * PC2_ROWS);
                tc::tma_load_2d_pair(buf + PC2_ROWS * ROWB, &mapA2, fb, x, (int)a2_row(0, row));
              } else {
                tc::tma_load_2d_pair(buf, &mapA2, fb, x, (int)a2_row(1, row));
                tc::tma_load_2d_pair(buf + G_BYTES, &mapA2, fb, x, (int)a2_row(2, row));
              }
              continue;
            }
            if (half == 0) {
              tc::mbar_expect_tx(&full[s], H1_BYTES);
              tc::tma_load_2d(buf, &mapG, &full[s], x, row);
#pragma unroll
              for (int b = 0; b < B1_NBOX; ++b)
                tc::tma_load_2d(buf + G_BYTES + b * B1_BOX * ROWB, &mapB1, &full[s], x, tt * B1_ROWS + b * B1_BOX);
            } else {
              const int y = (int)a2_row(0, row);
              tc::mbar_expect_tx(&full[s], H2_BYTES);
              tc::tma_load_2d(buf, &mapA2, &full[s], x, y);
              tc::tma_load_2d(buf + 3 * BM / 2 * ROWB, &mapA2, &full[s], x, y + 3 * BM / 2);
              tc::tma_load_2d(buf + 3 * G_BYTES, &mapB2, &full[s], x, tt * B2_ROWS);
            }
          }
        }
      }
      // the last release of every slot (ours and the peers') must land before we exit
      for (uint32_t s = 0; s < NSL && h > s; ++s) {
        const uint32_t uses = (h - s + NSL - 1) / NSL;
        tc::mbar_wait(&empty[s], (uses - 1) & 1, a.status, abort);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (PAIR && lane == 0 && leader) {
      constexpr uint32_t id256 = tc::idesc_bf16(2 * BM, 8 * TT), id64 = tc::idesc_bf16(2 * BM, 2 * TT);
      constexpr uint32_t id96 = tc::idesc_bf16(2 * BM, 3 * TT), id32 = tc::idesc_bf16(2 * BM, TT);
      constexpr uint32_t idI = tc::idesc_bf16(2 * BM, B1_ROWS <= 256 ? B1_ROWS : 256);
      constexpr uint32_t idF4 = tc::idesc_mxf4(2 * BM, B1_ROWS <= 256 ? B1_ROWS : 256);
      uint32_t h = 0, tcount = 0;
      bool ok = true;
      for (int u = cid; u < nsuper && ok; u += ncl, ++tcount) {
        const uint32_t ab = DB ? (tcount & 1) : 0, tacc = tbase + ab * 256;
        if ((DB ? tcount >= 2 : tcount > 0) &&
            !tc::mbar_wait(&acc_empty[ab], (DB ? (tcount >> 1) - 1 : tcount - 1) & 1, a.status, abort)) {
          ok = false;
          break;
        }
        tc::fence_after();
        for (int kb = 0; kb < nkb && ok; ++kb) {
          {
            // item 0: G and the C1 trait rows
            const uint32_t s = h % NSL;
            if (!tc::mbar_wait(&full[s], (h / NSL) & 1, a.status, abort)) { ok = false; break; }
            tc::fence_after();
            uint8_t* buf = smem + s * SLB;
            const uint64_t dg = tc::sdesc_sw128(buf), db = tc::sdesc_sw128(buf + G_BYTES);
            if (FP4) {
              // four K steps of 64 (32 bytes of each row), each digit into the same accumulator
              constexpr uint32_t sfb[3] = {SF_B0, SF_B1, SF_B2};
#pragma unroll
              for (int k = 0; k < BK4 / 64; ++k)
#pragma unroll
                for (int d = 0; d < 3; ++d)
                  tc::mma_mxf4_pair(tacc, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, d * F4_HALF * ROWB + k * 32), idF4,
                                    tbase + SF_A, tbase + sfb[d], (kb | k | d) ? 1u : 0u);
            } else {
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint32_t acc = (kb | k) ? 1u : 0u;
                if (INTERP) {
                  // one MMA over all C1 columns: each CTA supplies half of them, in the one-CTA order
                  tc::mma_bf16_pair(tacc, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, k * 32), idI, acc);
                } else {
                  // [Q1 | Q2] -> levels 0 and 1 of [w v1 v2 v3]; [Q3 | Q4] -> slices 3, 4 of w
                  tc::mma_bf16_pair(tbase + 0, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, k * 32), id256, acc);
                  tc::mma_bf16_pair(tbase + 8 * TT, tc::sdesc_add(dg, k * 32),
                                    tc::sdesc_add(db, 4 * TT * ROWB + k * 32), id64, acc);
                }
              }
            }
            tc::mma_commit_pair(&empty[s], (uint16_t)3);
            ++h;
          }
          if (!INTERP) {
            // items 1 and 2: the C2 trait rows and A1; A2 and A3s
            const uint32_t s1 = h % NSL, s2 = (h + 1) % NSL;
            if (!tc::mbar_wait(&full[s1], (h / NSL) & 1, a.status, abort) ||
                !tc::mbar_wait(&full[s2], ((h + 1) / NSL) & 1, a.status, abort)) {
              ok = false;
              break;
            }
            tc::fence_after();
            uint8_t* b1 = smem + s1 * SLB;
            uint8_t* b2 = smem + s2 * SLB;
            const uint64_t de = tc::sdesc_sw128(b1), d1 = tc::sdesc_sw128(b1 + PC2_ROWS * ROWB);
            const uint64_t d2 = tc::sdesc_sw128(b2), d3 = tc::sdesc_sw128(b2 + G_BYTES);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint32_t acc = (kb | k) ? 1u : 0u;
              tc::mma_bf16_pair(tbase + 10 * TT, tc::sdesc_add(d1, k * 32), tc::sdesc_add(de, k * 32), id96, acc);
              tc::mma_bf16_pair(tbase + 13 * TT, tc::sdesc_add(d2, k * 32),
                                tc::sdesc_add(de, (3 * TT / 2) * ROWB + k * 32), id64, acc);
              tc::mma_bf16_pair(tbase + 15 * TT, tc::sdesc_add(d3, k * 32),
                                tc::sdesc_add(de, (5 * TT / 2) * ROWB + k * 32), id32, acc);
            }
            tc::mma_commit_pair(&empty[s1], (uint16_t)3);
            tc::mma_commit_pair(&empty[s2], (uint16_t)3);
            h += 2;
          }
        }
        if (ok) tc::mma_commit_pair(&acc_full[ab], (uint16_t)3);
      }
    } else if (!PAIR && lane == 0) {
      constexpr uint32_t idN0 = tc::idesc_bf16(BM, N0), idN1 = tc::idesc_bf16(BM, N1 > 0 ? N1 : 16);
      constexpr uint32_t id3 = tc::idesc_bf16(BM, 3 * TT + C2_OFF), id2 = tc::idesc_bf16(BM, 2 * TT);
      constexpr uint32_t id1 = tc::idesc_bf16(BM, TT + C2_OFF);
      uint32_t h = 0, tcount = 0;
      bool ok = true;
      for (int u = cid; u < nsuper && ok; u += ncl, ++tcount) {
        const uint32_t ab = DB ? (tcount & 1) : 0, tacc = tbase + ab * 256;
        if ((DB ? tcount >= 2 : tcount > 0) &&
            !tc::mbar_wait(&acc_empty[ab], (DB ? (tcount >> 1) - 1 : tcount - 1) & 1, a.status, abort)) {
          ok = false;
          break;
        }
        tc::fence_after();
        for (int kb = 0; kb < nkb && ok; ++kb) {
          for (int half = 0; half < NI; ++half, ++h) {
            const uint32_t s = h % NSL;
            if (!tc::mbar_wait(&full[s], (h / NSL) & 1, a.status, abort)) { ok = false; break; }
            tc::fence_after();
            uint8_t* buf = smem + s * SLB;
            if (half == 0) {
              const uint64_t dg = tc::sdesc_sw128(buf);
              const uint64_t db = tc::sdesc_sw128(buf + G_BYTES);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint32_t acc = (kb | k) ? 1u : 0u;
                tc::mma_bf16(tacc, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, k * 32), idN0, acc);
                if (N1 > 0)
                  tc::mma_bf16(tacc + N0, tc::sdesc_add(dg, k * 32), tc::sdesc_add(db, N0 * ROWB + k * 32), idN1, acc);
              }
            } else {
              const uint64_t d1 = tc::sdesc_sw128(buf), d2 = tc::sdesc_sw128(buf + G_BYTES);
              const uint64_t d3 = tc::sdesc_sw128(buf + 2 * G_BYTES), de = tc::sdesc_sw128(buf + 3 * G_BYTES);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint32_t acc = (kb | k) ? 1u : 0u;
                // A1 x [E1 | E2 | E3s] -> [level 0 | a | b]  (8-trait tiles: [E2s | E1 | E2 | E3s])
                tc::mma_bf16(tbase + C2B, tc::sdesc_add(d1, k * 32), tc::sdesc_add(de, (TT - C2_OFF) * ROWB + k * 32),
                             id3, acc);
                // A2 x [E2s | E1] -> its own two groups
                tc::mma_bf16(tbase + C2B + C2_OFF + 3 * TT, tc::sdesc_add(d2, k * 32), tc::sdesc_add(de, k * 32), id2,
                             acc);
                // A3s x E1 -> its own group  (8-trait tiles: [E1 | E2])
                tc::mma_bf16(tbase + C2B + C2_OFF + 5 * TT, tc::sdesc_add(d3, k * 32),
                             tc::sdesc_add(de, TT * ROWB + k * 32), id1, acc);
              }
            }
            tc::mma_commit(&empty[s]);
          }
        }
        if (ok) tc::mma_commit(&acc_full[ab]);
      }
    }
  } else if (PSTAGE && warp == 2 + EPW) {
    // ------------------------------------------------------------ epilogue staging
    // tile k's data into buffer k & 1 once every epilogue warp is done with tile k - 2
    if (lane == 0) {
      uint32_t k = 0;
      for (int u = cid; u < nsuper; u += ncl, ++k) {
        if (k >= 2 && !tc::mbar_wait(&stage_empty[k & 1], ((k >> 1) - 1) & 1, a.status, abort)) break;
        issue_stage(u, (int)(k & 1));
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (EPW warps)
    const int ew = warp - 2;
    const int q = warp % 4;                            // TMEM lane quarter this warp may access
    constexpr int JPW = TT / (EPW / 4);                // traits per epilogue warp
    const int jbeg = (ew / 4) * JPW;
    const uint32_t lane_base = tbase + ((uint32_t)(q * 32) << 16);
    const float inv_dof = 1.f / a.dof;
    uint32_t tcount = 0;
    unsigned long long nsing = 0;
    for (int u = cid; u < nsuper; u += ncl, ++tcount) {
      // this tile's SNPs [snp0, snp0+128) (valid in [snp_lo, snp_end)), output origin and stride,
      // first trait (jbase) within its request, constants and output arrays
      int64_t snp0, snp_lo, snp_end, oi0, ldo;
      int ntrait, jbase, full_b;
      const float* cst_tile;
      float *obeta, *ose;
      double* ob64;
      unsigned long long* sing_ctr;
      if (SERVE) {
        const int4 w = a.units[u];
        const ServeDesc rd = a.reqs[w.z];
        snp0 = w.x; snp_lo = rd.i0; snp_end = rd.i1; oi0 = rd.i0; ldo = rd.ldo; ntrait = rd.ntrait; jbase = w.w * TT;
        full_b = rd.full_b; cst_tile = a.cst + (size_t)w.y * TT * CSTR;
        obeta = rd.beta; ose = rd.se; ob64 = rd.b64; sing_ctr = rd.singular;
      } else {
        int us, ut;
        super_coords<CS>(u, a, us, ut);
        const int st = us * CS + sr, tt = ut;
        snp0 = a.row0 + (int64_t)st * BM; snp_lo = a.snp_lo; snp_end = a.row0 + a.nsnp; oi0 = a.i0; ldo = a.ldo; ntrait = a.ntrait;
        jbase = tt * TT; full_b = a.full_b; cst_tile = a.cst + (size_t)jbase * CSTR;
        obeta = a.out_beta; ose = a.out_se; ob64 = a.out_b64; sing_ctr = nullptr;
      }
      // stage this tile's per-trait constants (double buffer: the barrier of the previous
      // tile guarantees every epilogue warp has finished reading this buffer)
      float* cs = cst_smem + (tcount & 1) * TT * CSTR;
      const float* ccur = PSTAGE ? cheb_c + (tcount & 1) * CBUF : cheb_c;
      const float* tcur = PSTAGE ? cheb_c + 2 * CBUF : cheb_t;
      bool staged = true;
      if (PSTAGE) {
        // this tile's bulk copies (issued during the tile before); T transposed for the series
        // (every warp passed barrier 2 of the previous tile, after its last read of the array)
        staged = tc::mbar_wait(&stage_full[tcount & 1], (tcount >> 1) & 1, a.status, abort);
        const float* tsrc = ccur + (CHEB_MAX_R + 1) * 128;
        float* tdst = cheb_c + 2 * CBUF;
        for (int e = ew * 32 + lane; e < a.cheb_R * TT; e += EPW * 32) tdst[e] = tsrc[(e % TT) * CHEB_MAX_R + e / TT];
        (void)cst_tile;
      } else {
      for (int e = ew * 32 + lane; e < TT * CSTR; e += EPW * 32)
        cs[e] = jbase + e / CSTR < ntrait ? cst_tile[e] : 0.f;
      }
      if (INTERP && !PSTAGE) {
        // the tile's Chebyshev coefficients (rows 0..R-1: c_k; row R: low part of c_0) and its
        // traits' T_k(x_j); one buffer: every warp passed barrier 2 of the previous tile, which
        // follows its last read of these
        const int R = a.cheb_R;
#pragma unroll 4
        for (int e = ew * 32 + lane; e < (R + 1) * 128; e += EPW * 32) {
          const int k = e >> 7, kk = k < R ? k : CHEB_MAX_R;
          cheb_c[e] = a.cheb_coef[(int64_t)kk * a.cheb_ld + snp0 + (e & 127)];
        }
        for (int e = ew * 32 + lane; e < R * TT; e += EPW * 32) {
          const int k = e / TT, jl = e % TT;
          cheb_t[e] = jbase + jl < ntrait ? a.cheb_T[(size_t)(jbase + jl) * CHEB_MAX_R + k] : 0.f;
        }
      }
      tc::named_sync(1, EPW * 32);
      const uint32_t ab = DB ? (tcount & 1) : 0;
      const bool ok = staged && tc::mbar_wait(&acc_full[ab], (DB ? tcount >> 1 : tcount) & 1, a.status, abort);
      const uint32_t lb = lane_base + ab * 256;  // this tile's accumulator buffer
      tc::fence_after();
      const int64_t snp = snp0 + q * 32 + lane;
      const bool valid_i = ok && snp >= snp_lo && snp < snp_end;
      const float sA = valid_i ? a.sA[snp] : 0.f;
      float ac[Q1] = {};
      if (valid_i && full_b == 1) {
#pragma unroll
        for (int c = 0; c < PM1; ++c) ac[c] = a.acoef[snp * PM1 + c];
      }
      unsigned long long tsing = 0;
      // All TMEM reads of this warp's JPW traits come first, reduced at once to the few
      // per-pair values the solve needs; the accumulators are released before any of the
      // per-pair arithmetic and output stores, so the next tile's MMAs wait only for the reads.
      static_assert(JPW % 4 == 0, "epilogue reads traits in groups of 4");
      float num_r[JPW], zz_r[JPW], s_r[JPW], z_r[JPW][Q1];
      const float F = 1.f / 256.f, FV = 1.f / 512.f;  // FV: the v' columns' second slice (9 bits)
#pragma unroll
      for (int g = 0; g < JPW / 4; ++g) {
        const int j0 = jbeg + 4 * g;
        {
          // C1, w: slices 1 and 2 (groups 0 and 1 + q) and the groups of slices 3 and 4 -> num
          uint32_t hw[4], lw[4], w3[4], w4[4];
          tc::tmem_ld4(lb + 0 * TT + j0, hw);
          tc::tmem_ld4(lb + (1 + PM1) * TT + j0, lw);
          tc::tmem_ld4(lb + (2 + 2 * PM1) * TT + j0, w3);
          tc::tmem_ld4(lb + (3 + 2 * PM1) * TT + j0, w4);
          tc::tmem_ld_wait();
          tc::reg_fence(hw); tc::reg_fence(lw); tc::reg_fence(w3); tc::reg_fence(w4);
          // two traits per packed instruction (each lane rounds as the scalar form would):
          // num = scale * (((w4 F + w3) F + lw) F + hw)
          const float2 F2 = make_float2(F, F);
#pragma unroll
          for (int v = 0; v < 4; v += 2) {
            float2 t = tc::ffma2(F2, make_float2(__uint_as_float(w4[v]), __uint_as_float(w4[v + 1])),
                                 make_float2(__uint_as_float(w3[v]), __uint_as_float(w3[v + 1])));
            t = tc::ffma2(F2, t, make_float2(__uint_as_float(lw[v]), __uint_as_float(lw[v + 1])));
            t = tc::ffma2(F2, t, make_float2(__uint_as_float(hw[v]), __uint_as_float(hw[v + 1])));
            const float2 nm = tc::fmul2(make_float2(cs[(j0 + v) * CSTR], cs[(j0 + v + 1) * CSTR]), t);
            num_r[4 * g + v] = nm.x;
            num_r[4 * g + v + 1] = nm.y;
            zz_r[4 * g + v] = 0.f;
            zz_r[4 * g + v + 1] = 0.f;
          }
        }
        // C1, v_c: slices 1 and 2 (groups 1 + c and 2 + q + c) -> z_c, three covariates per wait
#pragma unroll
        for (int c0 = 0; c0 < PM1; c0 += 3) {
          constexpr int CB = 3;
          uint32_t hz[CB][4], lz[CB][4];
#pragma unroll
          for (int c = 0; c < CB; ++c)
            if (c0 + c < PM1) {
              tc::tmem_ld4(lb + (1 + c0 + c) * TT + j0, hz[c]);
              tc::tmem_ld4(lb + (2 + PM1 + c0 + c) * TT + j0, lz[c]);
            }
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < CB; ++c)
            if (c0 + c < PM1) { tc::reg_fence(hz[c]); tc::reg_fence(lz[c]); }
          // z = scale * (lz FV + hz), zz += z^2, two traits per packed instruction
          const float2 FV2 = make_float2(FV, FV);
#pragma unroll
          for (int v = 0; v < 4; v += 2) {
            float2 zz2 = make_float2(zz_r[4 * g + v], zz_r[4 * g + v + 1]);
#pragma unroll
            for (int c = 0; c < CB; ++c)
              if (c0 + c < PM1) {
                const float2 z2 = tc::fmul2(
                    make_float2(cs[(j0 + v) * CSTR + 1 + c0 + c], cs[(j0 + v + 1) * CSTR + 1 + c0 + c]),
                    tc::ffma2(FV2, make_float2(__uint_as_float(lz[c][v]), __uint_as_float(lz[c][v + 1])),
                              make_float2(__uint_as_float(hz[c][v]), __uint_as_float(hz[c][v + 1]))));
                z_r[4 * g + v][c0 + c] = z2.x;
                z_r[4 * g + v + 1][c0 + c] = z2.y;
                zz2 = tc::ffma2(z2, z2, zz2);
              }
            zz_r[4 * g + v] = zz2.x;
            zz_r[4 * g + v + 1] = zz2.y;
          }
        }
        if (!INTERP) {
          // C2: level 0 and the five level-1 groups -> s
          uint32_t d0[4], da[4], db[4], ea[4], eb[4], ec[4];
          tc::tmem_ld4(lb + C2B + C2_OFF + 0 * TT + j0, d0);
          tc::tmem_ld4(lb + C2B + C2_OFF + 1 * TT + j0, da);
          tc::tmem_ld4(lb + C2B + C2_OFF + 2 * TT + j0, db);
          tc::tmem_ld4(lb + C2B + C2_OFF + 3 * TT + j0, ea);
          tc::tmem_ld4(lb + C2B + C2_OFF + 4 * TT + j0, eb);
          tc::tmem_ld4(lb + C2B + C2_OFF + 5 * TT + j0, ec);
          tc::tmem_ld_wait();
          tc::reg_fence(d0); tc::reg_fence(da); tc::reg_fence(db);
          tc::reg_fence(ea); tc::reg_fence(eb); tc::reg_fence(ec);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float lvl1 = (__uint_as_float(da[v]) + __uint_as_float(db[v])) +
                               (__uint_as_float(ea[v]) + __uint_as_float(eb[v])) + __uint_as_float(ec[v]);
            s_r[4 * g + v] = (sA * cs[(j0 + v) * CSTR + cst_escale(Q)]) * fmaf(F, lvl1, __uint_as_float(d0[v]));
            if (!SERVE && full_b == 2) {
              // node heritabilities of the interpolated S_BR: the two sums, combined in FP64 later
              const int jj = jbase + j0 + v;
              if (valid_i && jj < ntrait) {
                const int64_t o = (int64_t)jj * ldo + (snp - oi0);
                obeta[o] = __uint_as_float(d0[v]);
                ose[o] = lvl1;
              }
            }
          }
        }
      }
      // every TMEM read of this warp for this tile is complete: release the accumulators
      tc::fence_before();
      __syncwarp();
      if (lane == 0) {
        // relaxed: the TMEM loads are complete (tcgen05.wait::ld); nothing else is ordered
        if (PAIR) tc::mbar_arrive_cluster_relaxed(tc::mapa(&acc_empty[ab], 0));
        else tc::mbar_arrive(&acc_empty[ab]);
      }
      if (INTERP) {
        // S_BR = sum_k c_k T_k(x_j): the tail (k >= 2, terms decreasing like a geometric series)
        // in FP32 from the smallest term up, then c_0 (two floats) + c_1 T_1 (with the product's
        // rounding error) added last, so that s carries about one rounding of its own size
        const int R = a.cheb_R, i = q * 32 + lane;
        // two traits per packed FMA (each lane rounds as fmaf): the same sums, half the instructions
        float2 s2[JPW / 2];
#pragma unroll
        for (int r = 0; r < JPW / 2; ++r) s2[r] = make_float2(0.f, 0.f);
        for (int k = R - 1; k >= 2; --k) {
          const float ck = ccur[k * 128 + i];
          const float2 ck2 = make_float2(ck, ck);
#pragma unroll
          for (int r = 0; r < JPW / 2; ++r)
            s2[r] = tc::ffma2(ck2, *reinterpret_cast<const float2*>(tcur + k * TT + jbeg + 2 * r), s2[r]);
        }
#pragma unroll
        for (int r = 0; r < JPW / 2; ++r) {
          s_r[2 * r] = s2[r].x;
          s_r[2 * r + 1] = s2[r].y;
        }
        const float c0 = ccur[i], c1 = ccur[128 + i], c0lo = ccur[(PSTAGE ? CHEB_MAX_R : R) * 128 + i];
#pragma unroll
        for (int r = 0; r < JPW; ++r) {
          const float t1 = tcur[TT + jbeg + r];
          const float pp = c1 * t1, pe = fmaf(c1, t1, -pp);
          s_r[r] = c0 + (pp + ((s_r[r] + pe) + c0lo));
        }
        tc::named_sync(2, EPW * 32);
      }
      if (valid_i && full_b == 0) {
        // beta and SE of all the warp's traits first (independent chains that overlap), then the
        // stores of those in the block; the same operations per pair as below
        float beta_r[JPW], se_r[JPW];
        uint32_t singm = 0;
        // two traits per packed instruction where the operations allow it; each lane rounds as
        // the scalar tc::rcp_nr, products and FMAs would
#pragma unroll
        for (int r = 0; r < JPW; r += 2) {
          const float2 num = make_float2(num_r[r], num_r[r + 1]), s = make_float2(s_r[r], s_r[r + 1]);
          const float2 delta = make_float2(s.x - zz_r[r], s.y - zz_r[r + 1]);
          const bool sing0 = !(delta.x > 1e-6f * s.x) || !(sA > 0.f), sing1 = !(delta.y > 1e-6f * s.y) || !(sA > 0.f);
          const float2 y = make_float2(tc::rcp_approx(delta.x), tc::rcp_approx(delta.y));
          const float2 inv = tc::ffma2(y, tc::ffma2(make_float2(-delta.x, -delta.y), y, make_float2(1.f, 1.f)), y);
          const float2 beta = tc::fmul2(num, inv);
          const float2 rr = make_float2(cs[(jbeg + r) * CSTR + cst_rr(Q)], cs[(jbeg + r + 1) * CSTR + cst_rr(Q)]);
          const float2 rss0 = tc::ffma2(make_float2(-num.x, -num.y), beta, rr);
          const float2 rss = make_float2(fmaxf(rss0.x, 0.f), fmaxf(rss0.y, 0.f));
          const float2 x = tc::fmul2(tc::fmul2(rss, inv), make_float2(inv_dof, inv_dof));
          beta_r[r] = sing0 ? __int_as_float(0x7fc00000) : beta.x;
          beta_r[r + 1] = sing1 ? __int_as_float(0x7fc00000) : beta.y;
          se_r[r] = sing0 ? __int_as_float(0x7fc00000) : tc::sqrt_approx(x.x);
          se_r[r + 1] = sing1 ? __int_as_float(0x7fc00000) : tc::sqrt_approx(x.y);
          singm |= ((sing0 ? 1u : 0u) | (sing1 ? 2u : 0u)) << r;
        }
        const int nvalid = ntrait - (jbase + jbeg);
#pragma unroll
        for (int r = 0; r < JPW; ++r)
          if (r < nvalid) {
            const int64_t o = (int64_t)(jbase + jbeg + r) * ldo + (snp - oi0);
            // streaming stores: the grid is never re-read here, so it should not push the
            // genotype and trait tiles out of L2
            __stcs(obeta + o, beta_r[r]);
            __stcs(ose + o, se_r[r]);
            tsing += (singm >> r) & 1u;
          }
      }
      if (valid_i && full_b == 1) {
#pragma unroll
        for (int r = 0; r < JPW; ++r) {
          const int jl = jbeg + r;
          const int jj = jbase + jl;            // trait index within the block (request)
          if (jj >= ntrait) break;
          const float* cj = cs + jl * CSTR;
          const float num = num_r[r], zz = zz_r[r], s = s_r[r];
          const float delta = s - zz;
          float beta, se;
          const bool sing = !(delta > 1e-6f * s) || !(sA > 0.f);
          if (sing) {
            beta = se = __int_as_float(0x7fc00000);
            ++tsing;
          } else {
            const float inv = tc::rcp_nr(delta);
            beta = num * inv;
            const float rss = fmaxf(fmaf(-num, beta, cj[cst_rr(Q)]), 0.f);
            se = tc::sqrt_approx(rss * inv * inv_dof);
          }
          const int64_t o = (int64_t)jj * ldo + (snp - oi0);
          if (full_b == 1) {
            double* ob = ob64 + o * (PM1 + 1);
#pragma unroll
            for (int c = 0; c < PM1; ++c) {
              // beta_L = g - L^-T z beta - a_i beta
              float t = cj[cst_g(Q) + c];
#pragma unroll
              for (int d = 0; d < PM1; ++d) t = fmaf(-cj[cst_lit(Q) + c * PM1 + d] * z_r[r][d], beta, t);
              t = fmaf(-ac[c], beta, t);
              ob[c] = sing ? (double)beta : (double)t;
            }
            ob[PM1] = (double)beta;
          }
        }
      }
      if (PSTAGE) {
        // this warp's last read of the tile's staged data is done
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&stage_empty[tcount & 1]);
      }
      if (SERVE && sing_ctr) {
        unsigned long long v = tsing;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(sing_ctr, v);
      }
      nsing += tsing;
    }
    // warp-aggregated count of singular pairs
    for (int o = 16; o > 0; o >>= 1) nsing += __shfl_xor_sync(0xffffffffu, nsing, o);
    if (lane == 0 && nsing) atomicAdd(a.singular, nsing);
  }
  tc::fence_before();
  __syncthreads();
  if (PAIR) tc::cluster_sync();
  if (warp == 1) {
    if (PAIR) tc::tmem_dealloc_pair(tbase, TMEM_COLS);
    else tc::tmem_dealloc(tbase, TMEM_COLS);
  }
}

template <int EPW, bool SERVE, bool PAIR, int Q, bool INTERP = false, bool FP4 = false>
int launch_shape(gwas_ctx* c, const FusedArgs& a, const CUtensorMap& mg, const CUtensorMap& ma,
                 const CUtensorMap& m1, const CUtensorMap& m2) {
  constexpr int NC = PAIR ? 2 : 1;
  constexpr int SMEM = FP4 ? smem_bytes_fp4() : smem_bytes(PAIR, Q, INTERP);
  auto kern = fused_kernel<EPW, SERVE, PAIR, Q, INTERP, FP4>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(fused_threads(EPW, PAIR, INTERP));
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = c->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  int nclusters = nsm / NC;
  cfg.gridDim = dim3(nclusters * NC);
  int maxc = 0;
  if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) == cudaSuccess && maxc > 0) nclusters = maxc;
  cudaGetLastError();
  const int nsuper = SERVE ? a.nunits : ((a.n_stiles + NC - 1) / NC) * a.n_ttiles;
  nclusters = std::min(nclusters, nsuper);
  if (a.max_ctas > 0) nclusters = std::max(1, std::min(nclusters, a.max_ctas / NC));
  cfg.gridDim = dim3(nclusters * NC);
  ProfScope ps(c, SERVE ? "fused_serve" : a.full_b == 2 ? "cheb_nodes" : "fused");
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mg, ma, m1, m2, a);
  c->launches++;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, GWAS_ERR_CUDA, std::string("fused kernel launch: ") + cudaGetErrorString(e));
  }
  return GWAS_OK;
}

// Tensor maps of the one-CTA-per-tile shapes: boxes of 128 genotype rows, 192 rows of
// x'^2 planes, the C1 trait rows in one or two boxes of at most 256 rows, and the C2 trait rows.
bool make_big_maps(int q, CUtensorMap* mg, CUtensorMap* ma, CUtensorMap* m1, CUtensorMap* m2, const FusedArgs& a,
                   const __nv_bfloat16* G, const __nv_bfloat16* A2, const __nv_bfloat16* B1, const __nv_bfloat16* B2,
                   int ttiles) {
  const int r1 = c1_rows(q), r2 = c2_rows(q), b1box = r1 <= 256 ? r1 : r1 / 2;
  return make_bf16_map(mg, G, a.mpad, a.Kpad, BM, BK) && make_bf16_map(ma, A2, 3ull * a.mpad, a.Kpad, 3 * BM / 2, BK) &&
         make_bf16_map(m1, B1, (uint64_t)ttiles * r1, a.Kpad, b1box, BK) &&
         make_bf16_map(m2, B2, (uint64_t)ttiles * r2, a.Kpad, r2, BK);
}

}  // namespace
