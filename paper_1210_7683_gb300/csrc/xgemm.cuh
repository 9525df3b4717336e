// Exact sliced GEMM (see xgemm.cu): C[r][c] = sA[r] sB[c] sum_l 2^(-bits l) sum_{a+b=l} A_a[r] . B_b[c].
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

struct gwas_ctx;

struct XgemmArgs {
  int rows, cols;            // valid output rows (A rows) and columns (B rows)
  int rowsA_pad, rowsB_pad;  // plane row counts (multiples of 128 and 64)
  int Kpad;                  // K extent of the planes (multiple of 64), zero beyond the valid K
  double level_scale;        // 2^-bits
  const double* scaleA;      // per-row scale of A (NULL = 1)
  const double* scaleB;      // per-row scale of B
  double* out64;             // FP64 output (or NULL)
  float* out32;              // FP32 output when out64 is NULL
  int64_t ldo;               // output row stride (elements)
  unsigned long long* status;  // status[0] <- 1 when a bounded wait expires
  const char* name;          // timer name in profiling mode
  int untimed;               // nonzero: no timer of its own (the caller times an enclosing region)
  int kchunk;                // K chunk of one launch (multiple of 64; 0 = XGEMM_KCHUNK)
  int add_to_out;            // nonzero: the first chunk also adds to the output (out += A B^T)
  // set by launch_xgemm: the K blocks [kb0, kb1) of one launch, and whether it adds to the output
  int kb0, kb1, accumulate;
};

// K is contracted in chunks of at most XGEMM_KCHUNK; each chunk's level sums are exact
// in FP32 and the chunks are added in the output's precision.
constexpr int XGEMM_KCHUNK = 1024;

// Bits per slice for which the level-0 product of two slices is exact in FP32 over one
// K chunk: 2 * bits + log2(min(Kpad, XGEMM_KCHUNK)) <= 24 (7 bits for Kpad > 512).
inline int xgemm_bits(int Kpad) {
  const int K = Kpad < XGEMM_KCHUNK ? Kpad : XGEMM_KCHUNK;
  int lg = 0;
  while ((1 << lg) < K) ++lg;
  int b = (24 - lg) / 2;
  return b > 8 ? 8 : b;
}

// `name`: timer name in profiling mode (NULL: untimed, inside a region the caller times).
void launch_slice_rows(gwas_ctx* c, const double* src, int64_t lds, int rows, int K, int rows_pad, int Kpad, int S,
                       int bits, __nv_bfloat16* planes, double* scale, const char* name = "slice_rows");
// Instantiated slice configurations (SA, SB, L): (1, 4, 3) and (4, 4, 3), the 28-bit rotations,
// and (8, 8, 7), 56-bit operands for products accurate to FP64 (with kchunk <= 256 every level
// sum stays below 2^24 and is exact: 7-bit slices, |q_0| <= 2^7, |q_a| <= 2^6, so a level-l
// term is at most 2^12 (l + 3)).
int launch_xgemm(gwas_ctx* c, int SA, int SB, int L, const XgemmArgs& g, const __nv_bfloat16* A,
                 const __nv_bfloat16* B);
