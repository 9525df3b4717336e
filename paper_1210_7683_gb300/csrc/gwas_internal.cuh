// Internal declarations shared by the translation units of the GWAS library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/gwas.h"

#define GWAS_MAX_PM1 19

// Raw device buffer owned by a context; freed in gwas_destroy.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  bool pooled = false;  // from the library's device pool (else cudaMalloc)
};

struct MixedState;  // mixed-precision resident data (mixed.cu)
struct ServeState;  // serving scheduler (serve.cu)

// A kernel launch bracketed by two events on the context's stream (profiling mode).
struct ProfPending {
  const char* name;
  cudaEvent_t start, stop;
};

struct gwas_ctx {
  int n = 0, pm1 = 0, p = 0, t = 0, device = 0;
  int precision = GWAS_MIXED, output = GWAS_OUT_LAST_SE, trait_block = 0;
  size_t budget = 0, allocated = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<DevBuf> bufs;

  // preloop state (setup)
  double* Z = nullptr;     // n x n, column k = eigenvector k
  double* lam = nullptr;   // n eigenvalues, ascending
  double* XL = nullptr;    // [pm1][n]: row l = covariate l
  double* XLt = nullptr;   // [pm1][n]: row l = Z^T x_L,l
  double* h2 = nullptr;    // [t]
  std::vector<double> h_lam, h_h2;
  std::vector<double> h_XL;    // [pm1][n]
  std::vector<double> h_XtXinv;// (X_L^T X_L)^-1, pm1 x pm1

  // genotypes
  int64_t m = 0;
  double* Xt = nullptr;        // FP64 path: [m][n] rotated genotypes
  MixedState* mixed = nullptr; // mixed path state
  ServeState* serve = nullptr; // serving scheduler, started by the first gwas_submit

  // device status words: [0] timeout flag, [1..2] singular-pair counter (u64)
  unsigned long long* d_status = nullptr;
  int64_t singular = 0;
  int64_t launches = 0;
  int64_t fp4_launches = 0;  // launches of the fused kernel on e2m1 operands
  int eig_steps = -1;  // refinement steps of the eigendecomposition; -1: the FP64 solver computed it
  int64_t h2_gen = 0;  // incremented whenever the heritabilities change (gwas_set_h2)

  // output streaming: side stream and events of the double-buffered device-to-host copies
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_compute[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};

  // fused-kernel launch shape of the mixed path (from the autotuner or its cache; defaults otherwise):
  // CS x CT CTA clusters, EPW epilogue warps, CTA-pair mode, SNP tiles per traversal group
  struct FusedTune {
    int cs = 1, ct = 1, epw = 16, pair = 0, group = 16;
  } tune;
  std::string tune_cache;  // JSON cache of autotuned shapes ("" = none)

  // profiling: per-kernel device time from CUDA events on `stream`
  bool profile = false;
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::map<std::string, std::pair<double, int64_t>> prof;  // name -> (ms, launches)
};

// Brackets the kernel launches of its scope with events when profiling is on.
struct ProfScope {
  gwas_ctx* c;
  size_t idx;
  ProfScope(gwas_ctx* ctx, const char* name);
  ~ProfScope();
};
// Resolves the pending events (call after the stream has been synchronised).
void prof_flush(gwas_ctx* c);

// ---------------------------------------------------------------- helpers (api.cu)
// Restores the caller's current device when a call returns.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Applies the launch shape that c->tune_cache holds for this context's (n, p, mode, t), if any.
void tune_apply_cache(gwas_ctx* c);

// Phi = Z Lambda Z^T by the FP32 solver refined to FP64 accuracy (eig.cu): Z column-major, lam
// ascending, *steps = refinement steps taken.  Returns GWAS_OK, EIG_FALL_BACK when the FP64 solver
// must compute it instead (the FP32 solver failed, non-finite values, or no convergence), or an
// error code.  `solver` is the cusolverDnHandle_t, bound to c->stream.
constexpr int EIG_FALL_BACK = -1;
int eig_refined(gwas_ctx* c, void* solver, const double* phi, int n, double* Z, double* lam, int* steps);

int ctx_fail(gwas_ctx* c, int code, const std::string& msg);
int ctx_alloc(gwas_ctx* c, size_t bytes, void** out);          // budget-checked, from the device pool
void ctx_free(gwas_ctx* c, void* p);
bool ctx_cuda_ok(gwas_ctx* c, cudaError_t e, const char* what, int* rc);
// Copy `bytes` from a host or device pointer to a new or given device buffer.
int ctx_upload(gwas_ctx* c, const void* src, size_t bytes, void* dst);
int ptr_kind(gwas_ctx* c, const void* p, bool* is_device);

// ---------------------------------------------------------------- FP64 path (fp64.cu)
// C[r][col] = sum_k A[r][k] * Z[k][col] for r < rows, col < n (A row-major with leading dim lda).
void launch_rotate_fp64_i8(gwas_ctx* c, const int8_t* A, int64_t rows, int64_t lda, double* C);
void launch_rotate_fp64_f64(gwas_ctx* c, const double* A, int64_t rows, int64_t lda, double* C);
// Per-trait FP64 prep: R[j] = [e∘y~ | e∘x~_L | e] ([t][p+1][n]); consts[j] = {S_TL, b_T, yy}.
// X'_L = Z^T X_L for the few covariate rows (one warp per output).
void launch_rotate_fp64_rows(gwas_ctx* c, const double* A, int64_t rows, int64_t lda, double* C);
void launch_prep_fp64(gwas_ctx* c, const double* Yt, int tb, const double* h2, double* R, double* consts);
// Fused FP64 contraction + per-pair solve for SNPs [i0,i1) x traits [j0, j0+tb).
void launch_fused_fp64(gwas_ctx* c, int64_t i0, int64_t i1, int j0, int tb, int64_t ldo, const double* R,
                       const double* consts, void* out);
int consts_stride(int pm1);

// ---------------------------------------------------------------- mixed path (mixed.cu)
// Genotypes already on the device -> resident mixed-path arrays.  reuse: keep the arrays and
// the rotation scratch when they are large enough (out-of-core slabs), with no final
// synchronisation.
// `dXR`: device-readable genotypes; with `copy` (device, m x n) the conversion kernel, which reads
// them once, also writes them there and every later kernel reads the copy (dXR may then be mapped
// host memory).
int mixed_load(gwas_ctx* c, const int8_t* dXR, int64_t m, bool reuse = false, int8_t* copy = nullptr);
struct MixedWs;  // work buffers of one gwas_solve call (mixed.cu)
int mixed_ws_alloc(gwas_ctx* c, int tb_max, MixedWs** ws);
void mixed_ws_free(gwas_ctx* c, MixedWs* ws);
// Enqueues the per-trait operands of traits [0, tb) of dY (heritabilities h2, device) into
// trait tiles slot[j/32] (identity when slot is NULL) of the operand arrays B1, B2, cst, in the
// one-CTA layout or (pair != 0) the CTA-pair layout of the fused kernel.
// tt: trait-tile width of the C1 layout (0: mixed_tt; the interpolated kernel's tile_traits(q, true)).
// B1_4: the C1 operand as e2m1 digits instead of B1 (p = 4, interpolated 24-trait tiles, mixed_prep_block).
int mixed_prep_traits(gwas_ctx* c, MixedWs* ws, const double* dY, const double* h2, int tb, __nv_bfloat16* B1,
                      __nv_bfloat16* B2, float* cst, const int* slot, int pair, int tt = 0, uint8_t* B1_4 = nullptr);
// Enqueues (no synchronisation) the per-trait operands of traits [j0, j0+tb) into the workspace.
int mixed_prep_block(gwas_ctx* c, MixedWs* ws, const double* dY, int j0, int tb);
// Enqueues the fused kernel for the workspace's tb traits x SNPs [i0, i1) into dout.
int mixed_fused_block(gwas_ctx* c, MixedWs* ws, int tb, int64_t i0, int64_t i1, int64_t ldo, void* dout, int j0);
// The same for trait operands prepared elsewhere (mixed_prep_traits into B1, B2, cst).
// j0: the first trait of the block among the context's traits (its S_BR may then be interpolated
// in h^2), or -1 for traits with heritabilities of their own.
// B1_4: the C1 operand as e2m1 digits (then B1 is not read).
int mixed_fused_ops(gwas_ctx* c, const __nv_bfloat16* B1, const __nv_bfloat16* B2, const float* cst, int tb, int64_t i0,
                    int64_t i1, int64_t ldo, void* dout, int j0, const uint8_t* B1_4 = nullptr);
// Enqueues (no synchronisation) the solve of traits [j0, j0+tb) x SNPs [i0, i1) into dout.
int mixed_solve_block(gwas_ctx* c, MixedWs* ws, const double* dY, int j0, int tb, int64_t i0, int64_t i1, int64_t ldo,
                      void* dout);
void mixed_free(gwas_ctx* c);
void mixed_destroy(gwas_ctx* c);  // frees the mixed-path state itself (after mixed_free)
// S_BR by Chebyshev interpolation in h^2 over the context's heritabilities (mixed.cu): plans it
// for the current heritabilities (once per gwas_set_h2) and returns 1 when the kernel may use it,
// -1 when S_BR is contracted exactly.
int mixed_cheb_plan(gwas_ctx* c);
// State of the plan (1 usable, -1 exact, 0 not planned) with its terms, interval and error bound.
int mixed_cheb_info(gwas_ctx* c, int* R, double* lo, double* hi, double* bound);
// Whether the trait operands use the CTA-pair layout (the context's launch shape is the pair).
int mixed_pair_layout(gwas_ctx* c);
// Whether a block of tb of the context's traits runs the kernel with S_BR interpolated (tb > 1 and
// the plan allows it); its trait operands then use that kernel's layout (tile_traits(q, true)).
bool mixed_block_interp(gwas_ctx* c, int tb);
// resident mixed-path data (for the serving kernel launches)
int64_t mixed_mpad(gwas_ctx* c);
int mixed_kpad(gwas_ctx* c);  // padded n of the mixed path's operands (after mixed setup)
const float* mixed_sA(gwas_ctx* c);
const float* mixed_acoef(gwas_ctx* c);
const __nv_bfloat16* mixed_G(gwas_ctx* c);
const __nv_bfloat16* mixed_A2(gwas_ctx* c);
// 1 when the loaded genotypes also have their e2m1 copy (every value in {0, +-1, +-2, +-3, +-4, +-6})
// for the kernel on e2m1 operands
int mixed_fp4_ready(gwas_ctx* c);

// ---------------------------------------------------------------- serving (serve.cu)
void serve_shutdown(gwas_ctx* c);  // stops the scheduler thread and frees its memory
int serve_busy(gwas_ctx* c);       // requests queued or running
