// Fused contraction + Schur solve kernel (fused.cu).
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

struct gwas_ctx;

// Per-trait FP32 constants of the epilogue (stride FUSED_CST):
//   [0] scale of w, [1..3] scales of v'_1..3, [4] scale of e, [5] r^T M^-1 r,
//   [6..8] g = S_TL^-1 b_T, [9..17] L^-T (row-major), used for the full coefficient vector.
#define FUSED_CST 20

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
  int n_ttiles;       // ceil(ntrait / 32)
  int group;          // cluster-wide SNP super-tiles per traversal group (L2 reuse of genotype tiles)
  int ntrait;         // traits in this block
  int Kpad;           // padded n (multiple of 64)
  int64_t mpad;       // rows per plane of G and of the x'_c^2 planes
  float dof;          // n - p
  const float* sA;    // [m] scale of the x'_c^2 slices of each SNP (0 marks a singular SNP)
  const float* acoef; // [m][3] centring coefficients a_i (full output only)
  const float* cst;   // [ntrait][FUSED_CST]
  int full_b;         // 1: double b[ntrait][ldo][4]; 0: float beta/se [ntrait][ldo]
  int64_t ldo;        // output stride between traits (SNPs)
  float* out_beta;
  float* out_se;
  double* out_b64;
  unsigned long long* status;    // [0] <- 1 when a bounded wait expires
  unsigned long long* singular;  // singular-pair counter
  int max_ctas;       // 0 = one CTA per SM
  // serving mode: work units {first SNP row of the tile, trait-tile slot, request, request-local trait tile}
  const int4* units;
  int nunits;
  const ServeDesc* reqs;
};

// Trait operands (B1, B2) must be allocated (and zeroed) for a multiple of this many trait tiles,
// with 320 B1 rows and 192 B2 rows per trait tile.
int fused_trait_tile_multiple();
// 1 when the selected kernel shape is the CTA-pair one, whose trait operands use the pair layout.
int fused_pair_layout();

int launch_fused(gwas_ctx* c, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2);
// Serving mode: processes a.units (a.cst indexed by trait-tile slot) with per-request outputs.
// b_tiles = trait-tile slots of the B1/B2 arena.
int launch_fused_serve(gwas_ctx* c, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                       const __nv_bfloat16* B1, const __nv_bfloat16* B2, int b_tiles);
