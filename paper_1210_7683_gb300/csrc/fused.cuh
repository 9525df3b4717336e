// Fused contraction + Schur solve kernel (fused.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

struct gwas_ctx;

// Geometry of the mixed path for q = p - 1 covariates (0 <= q <= 19, i.e. 1 <= p <= 20).
//   A trait tile holds mixed_tt(q) traits.  Its C1 operand has c1_groups(q) groups of
//   mixed_tt(q) rows: [w1 | v_1..v_q] (slice 1), [w2 | v_1..v_q] (slice 2), w3, w4.  Its
//   C2 operand has 4 groups [E2s | E1 | E2 | E3s].  The accumulators of a tile take
//   c1_groups(q) * mixed_tt(q) + c2_cols(q) <= 512 TMEM columns, and the C1 half-stage (a
//   genotype tile and the C1 operand, 128-byte rows) fits a 64 KB ring slot.
__host__ __device__ constexpr int mixed_tt(int q) { return q <= 3 ? 32 : q <= 10 ? 16 : 8; }
__host__ __device__ constexpr int c1_groups(int q) { return 4 + 2 * q; }
__host__ __device__ constexpr int c1_rows(int q) { return c1_groups(q) * mixed_tt(q); }
__host__ __device__ constexpr int c2_rows(int q) { return 4 * mixed_tt(q); }
// TMEM columns of the C2 accumulators: six groups; with 8-trait tiles the MMAs (M = 128 needs
// N % 16 == 0) are widened to eight groups, two of which hold unused products.
__host__ __device__ constexpr int c2_cols(int q) { return mixed_tt(q) == 8 ? 8 * mixed_tt(q) : 6 * mixed_tt(q); }
// C2 rows allocated per trait tile (the CTA-pair layout, q = 3 only, needs 6 groups)
__host__ __device__ constexpr int c2_alloc(int q) { return 6 * mixed_tt(q); }
constexpr int MIXED_MAX_Q = 19;
// S_BR by Chebyshev interpolation in h^2: at most this many terms (node heritabilities).
constexpr int CHEB_MAX_R = 24;
// Trait-tile width of the kernel with S_BR interpolated: at q = 3 tiles of 24 traits, so that the
// C1 operand (10 groups, 240 rows) is one MMA of N <= 256 per K step and its accumulators can be
// double-buffered in TMEM; other q keep mixed_tt(q).  Its C1 operand is always in the one-CTA
// layout: the CTA pair splits that single MMA's rows in halves.
__host__ __device__ constexpr int tile_traits(int q, bool interp) { return interp && q == 3 ? 24 : mixed_tt(q); }
__host__ __device__ constexpr int c1_rows_of(int q, bool interp) { return c1_groups(q) * tile_traits(q, interp); }
// C1 operand rows to allocate for ntrait traits in either layout (trait tiles padded to a multiple of 4)
__host__ __device__ constexpr int64_t c1_alloc_rows(int q, int ntrait) {
  const int64_t a = ((ntrait + mixed_tt(q) - 1) / mixed_tt(q) + 3) / 4 * 4 * (int64_t)c1_rows(q);
  const int64_t b = ((ntrait + tile_traits(q, true) - 1) / tile_traits(q, true) + 3) / 4 * 4 * (int64_t)c1_rows_of(q, true);
  return a > b ? a : b;
}

// Runs the statement in the variadic arguments with the compile-time constant Q = q (0..7,
// larger values run as 7).
#define Q_DISPATCH(q, ...)                                   \
  switch (q) {                                               \
    case 0: { constexpr int Q = 0; __VA_ARGS__; } break;     \
    case 1: { constexpr int Q = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int Q = 2; __VA_ARGS__; } break;     \
    case 3: { constexpr int Q = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int Q = 4; __VA_ARGS__; } break;     \
    case 5: { constexpr int Q = 5; __VA_ARGS__; } break;     \
    case 6: { constexpr int Q = 6; __VA_ARGS__; } break;     \
    default: { constexpr int Q = 7; __VA_ARGS__; } break;    \
  }
// The same over 8..19 (smaller values run as 8).
#define Q_DISPATCH_WIDE(q, ...)                              \
  switch (q) {                                               \
    case 9: { constexpr int Q = 9; __VA_ARGS__; } break;     \
    case 10: { constexpr int Q = 10; __VA_ARGS__; } break;   \
    case 11: { constexpr int Q = 11; __VA_ARGS__; } break;   \
    case 12: { constexpr int Q = 12; __VA_ARGS__; } break;   \
    case 13: { constexpr int Q = 13; __VA_ARGS__; } break;   \
    case 14: { constexpr int Q = 14; __VA_ARGS__; } break;   \
    case 15: { constexpr int Q = 15; __VA_ARGS__; } break;   \
    case 16: { constexpr int Q = 16; __VA_ARGS__; } break;   \
    case 17: { constexpr int Q = 17; __VA_ARGS__; } break;   \
    case 18: { constexpr int Q = 18; __VA_ARGS__; } break;   \
    case 19: { constexpr int Q = 19; __VA_ARGS__; } break;   \
    default: { constexpr int Q = 8; __VA_ARGS__; } break;    \
  }
// Q = q for 0 <= q <= 19.
#define Q_DISPATCH_ALL(q, ...)                               \
  if ((q) <= 7) {                                            \
    Q_DISPATCH(q, __VA_ARGS__)                               \
  } else {                                                   \
    Q_DISPATCH_WIDE(q, __VA_ARGS__)                          \
  }

// Per-trait FP32 constants of the epilogue, cst_stride(q) floats per trait:
//   [0] scale of w, [1..q] scales of v'_1..q, [q+1] scale of e, [q+2] r^T M^-1 r,
//   [q+3 .. 2q+2] g = S_TL^-1 b_T, [2q+3 ..] L^-T (q x q, row-major), used for the full
//   coefficient vector.
__host__ __device__ constexpr int cst_stride(int q) { return (3 + 2 * q + q * q + 3) / 4 * 4; }
__host__ __device__ constexpr int cst_escale(int q) { return q + 1; }
__host__ __device__ constexpr int cst_rr(int q) { return q + 2; }
__host__ __device__ constexpr int cst_g(int q) { return q + 3; }
__host__ __device__ constexpr int cst_lit(int q) { return 2 * q + 3; }
static_assert(cst_stride(3) == 20 && c1_rows(3) + c2_cols(3) == 512, "p = 4 geometry");
__host__ __device__ constexpr bool tmem_fits_all_q() {
  for (int q = 0; q <= MIXED_MAX_Q; ++q)
    if (c1_rows(q) + c2_cols(q) > 512 || c1_rows(q) % 16 || c2_cols(q) % 16) return false;
  return true;
}
static_assert(tmem_fits_all_q(), "TMEM columns");

// Row of plane p (0..2) of SNP i in the x'_c^2 slice array: the three planes of each
// 128-SNP tile are stored next to one another ([tile][plane][128 rows][Kpad]), so that
// one tile's planes are 384 consecutive rows and load as two large TMA boxes.
__host__ __device__ __forceinline__ int64_t a2_row(int p, int64_t i) { return ((i >> 7) * 3 + p) * 128 + (i & 127); }

// Serving mode: one request of the work list (fused.cu, serve.cu).
struct ServeDesc {
  int64_t i0, i1;     // SNP range of the request
  int64_t ldo;        // output stride between traits (= i1 - i0)
  int ntrait;         // traits of the request
  int full_b;
  float* beta;        // LAST_SE outputs (device or page-locked host memory)
  float* se;
  double* b64;        // FULL_B output
  unsigned long long* singular;  // per-request singular-pair counter
};

struct FusedArgs {
  int64_t row0;       // first SNP of the first tile (a multiple of 128)
  int64_t snp_lo;     // first SNP of the range (row0 <= snp_lo < row0 + 128); SNPs below it are not written
  int64_t i0;         // SNP index that maps to output column 0
  int64_t nsnp;       // SNPs from row0 to the end of the range
  int n_stiles;       // ceil(nsnp / 128)
  int n_ttiles;       // ceil(ntrait / mixed_tt(q))
  int group;          // cluster-wide SNP super-tiles per traversal group (L2 reuse of genotype tiles)
  int ntrait;         // traits in this block
  int Kpad;           // padded n (multiple of 64)
  int Kp4;            // padded n of the e2m1 operands (multiple of 256; FP4 kernel only)
  int64_t mpad;       // rows per plane of G and of the x'_c^2 planes
  float dof;          // n - p
  const float* sA;    // [m] scale of the x'_c^2 slices of each SNP (0 marks a singular SNP)
  const float* acoef; // [m][q] centring coefficients a_i (full output only)
  const float* cst;   // [trait tiles * mixed_tt(q)][cst_stride(q)]
  int full_b;         // 1: double b[ntrait][ldo][q + 1]; 0: float beta/se [ntrait][ldo];
                      // 2: the level-0 and level-1 sums of S_BR into out_beta / out_se [ntrait][ldo]
                      //    (node heritabilities of the Chebyshev interpolation; exact kernel only)
  int64_t ldo;        // output stride between traits (SNPs)
  float* out_beta;
  float* out_se;
  double* out_b64;
  unsigned long long* status;    // [0] <- 1 when a bounded wait expires
  unsigned long long* singular;  // singular-pair counter
  int max_ctas;       // 0 = one CTA per SM
  // serving mode: work units {first SNP row of the tile, trait-tile slot, request, request-local trait tile}
  const int4* units;
  int nunits;             // units (an upper bound when nunits_dev is set)
  const int* nunits_dev;  // NULL, or the units of the launch in device memory (captured graphs)
  const ServeDesc* reqs;
  // S_BR by Chebyshev interpolation in h^2 (NULL cheb_coef: S_BR is contracted in the kernel):
  // s_ij = sum_{k < cheb_R} c_ik T_k(x_j), c_ik = cheb_coef[k * cheb_ld + i] (row CHEB_MAX_R
  // holds the low part of c_i0), T_k(x_j) = cheb_T[j * CHEB_MAX_R + k] for the block's trait j
  const float* cheb_coef;
  const float* cheb_T;
  int cheb_R;
  int64_t cheb_ld;
};

// Trait operands (B1, B2) must be allocated (and zeroed) for a multiple of this many trait tiles,
// with c1_rows(q) B1 rows and c2_alloc(q) B2 rows per trait tile.
int fused_trait_tile_multiple();
// 1 when the context's kernel shape is the CTA-pair one, whose trait operands use the pair layout.
int fused_pair_layout(const gwas_ctx* c, int q);
// Whether a launch shape (CS x CT cluster, EPW epilogue warps, CTA pair) is built for q.
bool fused_shape_supported(int q, int cs, int ct, int epw, int pair);

// q = p - 1 (0..19) selects the kernel's geometry; shapes other than the default one-CTA
// shape are built for q = 3 only.
int launch_fused(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2);
// The kernel with S_BR evaluated from its Chebyshev series in h^2 (a.cheb_coef set):
// 0 <= q <= 7 in fused_cheb.cu, 8 <= q <= 19 in fused_cheb_wide.cu; b_tiles as above.
int launch_fused_cheb(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* B1,
                      int b_tiles);
int launch_fused_cheb_wide(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* B1,
                           int b_tiles);
// The CTA-pair shape of the same (q = 3, trait operands in the pair layout).
int launch_fused_cheb_pair(gwas_ctx* c, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* B1,
                           int b_tiles);
// The CTA-pair shape with S_BR interpolated on e2m1 operands (fused_fp4.cu, q = 3): G4 the
// genotypes [mpad][Kp4 / 2] (two e2m1 values per byte), B1_4 the C1 trait columns as three
// e2m1 digits per fixed-point slice, [trait tile][CTA half][digit][120 rows][Kp4 / 2].  The
// accumulators hold the same integers as the bf16 kernel's, so the outputs are the same.
int launch_fused_cheb_pair_fp4(gwas_ctx* c, const FusedArgs& a, const uint8_t* G4, const uint8_t* B1_4, int b_tiles);
// Rows of B1_4 per trait tile: 3 digits x the 240 C1 rows of a 24-trait tile.
constexpr int FP4_TILE_ROWS = 3 * 240;
// Single-trait kernel (gemv.cu): the same solve for a.ntrait == 1, streaming the SNPs'
// operands once through a TMA ring (HBM-bound); for the one-CTA operand layout, 0 <= q <= 19.
bool gemv1_supported(int q, int Kpad);
// 8 <= q <= 19 (gemv_wide.cu), with the tensor maps launch_gemv1 builds.
int launch_gemv1_wide(gwas_ctx* c, int q, const FusedArgs& a, const CUtensorMap& mg, const CUtensorMap& ma,
                      const CUtensorMap& m1, const CUtensorMap& m2);
int launch_gemv1(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2);
// Serving mode: processes a.units (a.cst indexed by trait-tile slot) with per-request outputs.
// b_tiles = trait-tile slots of the B1/B2 arena.
int launch_fused_serve(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                       const __nv_bfloat16* B1, const __nv_bfloat16* B2, int b_tiles);
// The one-CTA kernel for 8 <= q <= 19 (fused_wide.cu), for either of the two launches above;
// b_tiles = trait tiles allocated in B1/B2.
int launch_fused_wide(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                      const __nv_bfloat16* B1, const __nv_bfloat16* B2, bool serve, int b_tiles);
