// Exact sliced GEMM on the tensor cores (the error-free splitting of Ozaki, Ogita,
// Oishi and Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication", 2012, in fixed-point form).
//
// Each operand row is written as  x = s * sum_a q_a 2^(-bits*a)  with integer
// slices |q_a| <= 2^bits (exact in bf16) and a per-row scale s.  The product
// C = A B^T is assembled from the slice products A_a B_b^T with a + b <= L; all
// products of one level a + b share a TMEM accumulator.  Level 0 is a single
// product whose partial sums stay below 2^24 (2*bits + log2(K) <= 24), so it is
// exact in FP32 whatever the accumulation order; the higher levels are 2^-bits
// smaller and their FP32 rounding is negligible.  The epilogue combines the
// levels and the scales in FP64.  K is contracted in chunks of at most 1024, one launch
// each, so that bits = 7 at any n (4 slices: 28 bits); later chunks add to the output.
//
// Used for the rotations by Z of Algorithm 5 (X'_R := Z^T X_R with exact int8
// genotypes as A, and Y' := Z^T Y) and for the back-rotation Z W' of the
// per-trait operands, with 4 slices of 7 bits; and with 8 slices and K chunks of
// 256 for the FP64-accurate products of the eigendecomposition's refinement (eig.cu).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <memory>

#include "gwas_internal.cuh"
#include "tc.cuh"
#include "xgemm.cuh"

namespace {

constexpr int BM = 128, BK = 64;

template <int SA, int SB, int L>
struct XCfg {
  // wider N when A has a single slice: (L+1) accumulators of BN columns fit TMEM
  static constexpr int BN = (SA == 1 && (L + 1) * 128 <= 512) ? 128 : 64;
  static constexpr int A_BYTES = BM * BK * 2;            // one slice plane tile
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = SA * A_BYTES + SB * B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE >= 4 ? 4 : (200 * 1024) / STAGE;
  static constexpr int TMEM_COLS = (L + 1) * BN <= 128 ? 128 : ((L + 1) * BN <= 256 ? 256 : 512);
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

template <int SA, int SB, int L>
__global__ void __launch_bounds__(192, 1) xgemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                       const __grid_constant__ CUtensorMap mapB, XgemmArgs g) {
  using Cfg = XCfg<SA, SB, L>;
  constexpr int BN = Cfg::BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + Cfg::STAGES * Cfg::STAGE);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* done = empty + Cfg::STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // column tiles along x: the CTAs of one row tile are scheduled together and share its A tile in L2
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const int kb0 = g.kb0, nk = g.kb1 - g.kb0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tslot, Cfg::TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0 && lane == 0) {
    tc::prefetch_map(&mapA);
    tc::prefetch_map(&mapB);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % Cfg::STAGES;
      if (kb >= Cfg::STAGES && !tc::mbar_wait(&empty[s], ((kb / Cfg::STAGES) - 1) & 1, g.status, abort)) break;
      uint8_t* st = smem + s * Cfg::STAGE;
      tc::mbar_expect_tx(&full[s], Cfg::STAGE);
#pragma unroll
      for (int a = 0; a < SA; ++a)
        tc::tma_load_2d(st + a * Cfg::A_BYTES, &mapA, &full[s], (kb0 + kb) * BK, a * g.rowsA_pad + r0);
#pragma unroll
      for (int b = 0; b < SB; ++b)
        tc::tma_load_2d(st + SA * Cfg::A_BYTES + b * Cfg::B_BYTES, &mapB, &full[s], (kb0 + kb) * BK,
                        b * g.rowsB_pad + c0);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16(BM, BN);
    bool ok = true;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % Cfg::STAGES;
      if (!tc::mbar_wait(&full[s], (kb / Cfg::STAGES) & 1, g.status, abort)) { ok = false; break; }
      tc::fence_after();
      uint8_t* st = smem + s * Cfg::STAGE;
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        bool first[L + 1];
#pragma unroll
        for (int l = 0; l <= L; ++l) first[l] = (kb == 0 && k == 0);
#pragma unroll
        for (int a = 0; a < SA; ++a)
#pragma unroll
          for (int b = 0; b < SB; ++b) {
            if (a + b > L) continue;
            const uint64_t ad = tc::sdesc_add(tc::sdesc_sw128(st + a * Cfg::A_BYTES), k * 32);
            const uint64_t bd = tc::sdesc_add(tc::sdesc_sw128(st + SA * Cfg::A_BYTES + b * Cfg::B_BYTES), k * 32);
            tc::mma_bf16(tbase + (a + b) * BN, ad, bd, idesc, first[a + b] ? 0u : 1u);
            first[a + b] = false;
          }
      }
      tc::mma_commit(&empty[s]);
    }
    tc::mma_commit(done);
  } else if (warp >= 2) {
    const int q = warp % 4;
    const bool ok = tc::mbar_wait(done, 0, g.status, abort);
    tc::fence_after();
    const int r = r0 + q * 32 + lane;
    const double sa = (ok && r < g.rows) ? (g.scaleA ? g.scaleA[r] : 1.0) : 0.0;
    // level_scale = 2^-bits: the value of levels 0..3 is hi * 2^(-bits min(L, 3)), that of levels
    // 4..L is lo * 2^(-bits L)
    const int bits = -ilogb(g.level_scale);
    const double hi_scale = ldexp(1.0, -bits * (L < 3 ? L : 3));
    const double lo_scale = ldexp(1.0, -bits * (L > 3 ? L - 3 : 0));
    for (int cc = 0; cc < BN; cc += 8) {
      uint32_t v[L + 1][8];
#pragma unroll
      for (int l = 0; l <= L; ++l) tc::tmem_ld8(tbase + ((uint32_t)(q * 32) << 16) + l * BN + cc, v[l]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int l = 0; l <= L; ++l) tc::reg_fence(v[l]);
      if (!ok || r >= g.rows) continue;
      if (g.out64) {
        // Every level sum is an integer held exactly by its FP32 accumulator (|sum| < 2^26), so
        // the levels are converted to 32-bit integers and combined exactly in 64-bit integers,
        // levels 0..3 and 4..7 apart (bits <= 8 keeps each group below 2^53), then converted to
        // FP64 once per group: FP64, and conversions to or from 64-bit types, run at a small
        // fraction of the 32-bit rates on this GPU.
        constexpr int H = L < 3 ? L : 3;
        const long long base = 1LL << bits;
        const double sah = sa * hi_scale;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = c0 + cc + j;
          if (c >= g.cols) break;
          long long hi = 0;
#pragma unroll
          for (int l = 0; l <= H; ++l) hi = hi * base + __float2int_rn(__uint_as_float(v[l][j]));
          double acc = (double)hi;
          if constexpr (L > 3) {
            long long lo = 0;
#pragma unroll
            for (int l = 4; l <= L; ++l) lo = lo * base + __float2int_rn(__uint_as_float(v[l][j]));
            acc = fma((double)lo, lo_scale, acc);
          }
          double* o = g.out64 + (size_t)r * g.ldo + c;
          const double val = acc * (sah * g.scaleB[c]);
          *o = g.accumulate ? *o + val : val;
        }
      } else {
        // FP32 result: each level sum is an exact integer below 2^24, so combining the
        // levels in FP32 (smallest first) costs no more than the final rounding
        const float ls = (float)g.level_scale, saf = (float)sa;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = c0 + cc + j;
          if (c >= g.cols) break;
          float acc = __uint_as_float(v[L][j]);
#pragma unroll
          for (int l = L - 1; l >= 0; --l) acc = fmaf(acc, ls, __uint_as_float(v[l][j]));
          float* o = g.out32 + (size_t)r * g.ldo + c;
          *o = g.accumulate ? *o + acc * (saf * (float)g.scaleB[c]) : acc * (saf * (float)g.scaleB[c]);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, Cfg::TMEM_COLS);
}

// ------------------------------------------------------------------ row slicing
// Slices of each row of a FP64 matrix (row r at src + r*lds, K valid entries) into
// S bf16 planes [S][rows_pad][Kpad]: x = scale * sum_a q_a 2^(-bits a), scale =
// max|x| / 2^bits, q_0 in [-2^bits, 2^bits], later |q_a| <= 2^(bits-1).
//
// The digits come from one 64-bit fixed-point integer per element,
// X = round(x / scale * 2^(bits (S-1))), |X| <= 2^(bits S): q_0 = round(X / 2^(bits (S-1))), and
// each later digit is the rounded quotient of the remainder by the next power 2^(bits (S-1-a)),
// so every remainder is at most half that power.  Two FP64 operations per element (the scaling
// and the conversion) instead of three per digit; the digits and the dropped tail are those of
// rounding digit by digit.  bits * S > 62 (not used by this library) takes the FP64 loop.
// Row maxima compare the bit patterns of |x| as integers (order-preserving for non-negative
// doubles).  A non-finite entry gives NaN slices.
__global__ void slice_rows_kernel(const double* __restrict__ src, int64_t lds, int rows, int K, int rows_pad, int Kpad,
                                  int S, int bits, __nv_bfloat16* __restrict__ planes, double* __restrict__ scale) {
  const int warps = blockDim.x / 32;
  const int r = blockIdx.x * warps + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (r >= rows_pad) return;
  const double* row = src + (size_t)r * lds;
  unsigned long long mb = 0;
  if (r < rows)
    for (int k = lane; k < K; k += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(row[k]) & 0x7fffffffffffffffULL;
      mb = b > mb ? b : mb;
    }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = b > mb ? b : mb;
  }
  const double mx = __longlong_as_double((long long)mb);
  const double s = (mx > 0 && mx <= 1.7976931348623157e308) ? ldexp(mx, -bits) : 1.0;
  if (lane == 0 && r < rows) scale[r] = s;
  const size_t plane = (size_t)rows_pad * Kpad;
  __nv_bfloat16* out = planes + (size_t)r * Kpad;
  const int top = bits * (S - 1);
  const double inv = ldexp(1.0 / s, top);  // 2^top / scale
  if (bits * S <= 62 && isfinite(inv)) {
    for (int k = lane; k < Kpad; k += 32) {
      const double x = (r < rows && k < K) ? row[k] : 0.0;
      if (!isfinite(x)) {
        for (int a = 0; a < S; ++a) out[a * plane + k] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
        continue;
      }
      long long X = __double2ll_rn(x * inv);
      for (int a = 0; a < S; ++a) {
        const int sh = top - bits * a;
        const long long q = sh > 0 ? ((X + (1LL << (sh - 1))) >> sh) : X;
        X -= q * (1LL << sh);
        out[a * plane + k] = __float2bfloat16_rn((float)(int)q);
      }
    }
  } else {
    const double two = ldexp(1.0, bits), inv = 1.0 / s;
    for (int k = lane; k < Kpad; k += 32) {
      double x = (r < rows && k < K) ? row[k] * inv : 0.0;
      for (int a = 0; a < S; ++a) {
        const double q = rint(x);
        out[a * plane + k] = __double2bfloat16(q);
        x = (x - q) * two;
      }
    }
  }
}

}  // namespace

bool make_bf16_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows,
                   uint32_t box_cols) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    enc = (EncodeFn)fn;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_bf16_map_strided(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t row_stride,
                           uint32_t box_rows, uint32_t box_cols) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {row_stride * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t es[2] = {1, 1};
  return ((EncodeFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_f32_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows,
                  uint32_t box_cols) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 4};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t es[2] = {1, 1};
  return ((EncodeFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_u8_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols};
  cuuint32_t box[2] = {128, box_rows};
  cuuint32_t es[2] = {1, 1};
  return ((EncodeFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_slice_rows(gwas_ctx* c, const double* src, int64_t lds, int rows, int K, int rows_pad, int Kpad, int S,
                       int bits, __nv_bfloat16* planes, double* scale, const char* name) {
  const int warps = 8;
  std::unique_ptr<ProfScope> ps(name ? new ProfScope(c, name) : nullptr);
  slice_rows_kernel<<<(rows_pad + warps - 1) / warps, warps * 32, 0, c->stream>>>(src, lds, rows, K, rows_pad, Kpad, S,
                                                                                  bits, planes, scale);
  c->launches++;
}

template <int SA, int SB, int L>
static int run_xgemm(gwas_ctx* c, const XgemmArgs& g, const __nv_bfloat16* A, const __nv_bfloat16* B) {
  using Cfg = XCfg<SA, SB, L>;
  CUtensorMap ma, mb;
  if (!make_bf16_map(&ma, A, (uint64_t)SA * g.rowsA_pad, g.Kpad, BM) ||
      !make_bf16_map(&mb, B, (uint64_t)SB * g.rowsB_pad, g.Kpad, Cfg::BN))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(xgemm_kernel<SA, SB, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    attr = true;
  }
  // a last partial column tile reads past its plane (the next plane, or TMA zero fill
  // after the last one); those columns are >= g.cols and never stored
  dim3 grid((g.rowsB_pad + Cfg::BN - 1) / Cfg::BN, g.rowsA_pad / BM);
  if (grid.y > 65535) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "xgemm: more than 65535 row tiles");
  std::unique_ptr<ProfScope> ps(g.untimed ? nullptr : new ProfScope(c, g.name ? g.name : "xgemm"));
  xgemm_kernel<SA, SB, L><<<grid, 192, Cfg::SMEM, c->stream>>>(ma, mb, g);
  c->launches++;
  return GWAS_OK;
}

int launch_xgemm(gwas_ctx* c, int SA, int SB, int L, const XgemmArgs& args, const __nv_bfloat16* A,
                 const __nv_bfloat16* B) {
  if (args.rowsA_pad % BM || args.rowsB_pad % 64 || args.Kpad % BK)
    return ctx_fail(c, GWAS_ERR_ARG, "xgemm: padded sizes are not tile multiples");
  if (!((SA == 4 && SB == 4 && L == 3) || (SA == 1 && SB == 4 && L == 3) || (SA == 8 && SB == 8 && L == 7)))
    return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "xgemm: slice configuration not instantiated");
  const int chunk = args.kchunk > 0 ? args.kchunk : XGEMM_KCHUNK;
  if (chunk % BK || chunk > XGEMM_KCHUNK) return ctx_fail(c, GWAS_ERR_ARG, "xgemm: bad K chunk");
  for (int k0 = 0; k0 < args.Kpad; k0 += chunk) {
    XgemmArgs g = args;
    g.kb0 = k0 / BK;
    g.kb1 = std::min(args.Kpad, k0 + chunk) / BK;
    g.accumulate = k0 > 0 || args.add_to_out;
    const int rc = SA == 8   ? run_xgemm<8, 8, 7>(c, g, A, B)
                   : SA == 4 ? run_xgemm<4, 4, 3>(c, g, A, B)
                             : run_xgemm<1, 4, 3>(c, g, A, B);
    if (rc != GWAS_OK) return rc;
  }
  return GWAS_OK;
}
