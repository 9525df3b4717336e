/*
 * gwas.h -- C interface of the GB300 multi-trait GWAS library.
 *
 * The library solves the m x t grid of generalized least-squares problems of
 * Section 2, Eq. (1):
 *
 *     b_ij = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j,
 *     X_i  = [X_L | x_i]            (X_L: n x (p-1) covariates, x_i: SNP i),
 *     M_j  = h_j^2 Phi + (1 - h_j^2) I                               (Eq. 2),
 *
 * by the eigendecomposition method of Section 3 (Algorithm 5): one FP64
 * eigendecomposition Phi = Z Lambda Z^T, a rotation of genotypes and traits
 * by Z^T, and, per (SNP, trait) pair, dense contractions over n followed by
 * a p x p solve.  The scale sigma_j^2 of Eq. (2) does not change b_ij nor
 * the standard error and is not an input.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major.  X_R (genotypes) is n x m int8, i.e. SNP-major:
 *   the n genotypes of SNP i are contiguous.  Y is n x t FP64: the n values of
 *   trait j are contiguous.
 * - Every array argument may be a host pointer (pageable or pinned) or a device
 *   pointer on the context's device; the library tells them apart with
 *   cudaPointerGetAttributes and copies host data itself (where the device reads
 *   the CPU's page tables, kernels read page-locked genotypes and store
 *   page-locked outputs directly instead).  The caller keeps ownership of all
 *   its buffers and may release them when the call returns.
 * - The context owns every device allocation it makes (Z, Lambda, the rotated
 *   covariates, the resident rotated genotypes and the work buffers) and gives
 *   them back in gwas_destroy to the library's device memory pool, which keeps
 *   them for the next context (gwas_pool_info, gwas_pool_trim).
 * - Calls on one context are not thread-safe; different contexts are
 *   independent.  All work runs on the context's stream; calls return after
 *   their results are complete (host outputs written, device outputs ready).
 * - Every call returns a status code; on failure gwas_last_error() returns a
 *   one-line description.  A failed call leaves previously loaded state valid
 *   unless the message says otherwise.
 */
#ifndef GWAS_GB300_H
#define GWAS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GWAS_API __attribute__((visibility("default")))
#else
#define GWAS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GWAS_OK                 0
#define GWAS_ERR_ARG            1  /* invalid argument (size, range, pointer on another device) */
#define GWAS_ERR_NOT_SPD        2  /* some M_j is not positive definite, or the eigensolver failed */
#define GWAS_ERR_OOM            3  /* the request exceeds the HBM budget or a device allocation failed */
#define GWAS_ERR_CUDA           4  /* a CUDA runtime or library call failed */
#define GWAS_ERR_TIMEOUT        5  /* a bounded wait inside a kernel ran out; results are invalid */
#define GWAS_ERR_SINGULAR_PAIRS 6  /* warning: some pairs have a (numerically) singular p x p system;
                                      their outputs are NaN, every other output is valid */
#define GWAS_ERR_STATE          7  /* call out of order (e.g. gwas_solve before gwas_load_snps) */
#define GWAS_ERR_UNSUPPORTED    8  /* a size or mode the library does not implement */

/* precision modes */
#define GWAS_FP64  0  /* every step in FP64 (the paper's arithmetic, Section 6) */
#define GWAS_MIXED 1  /* bf16 tensor-core contractions on exact fixed-point slices with
                         FP32 accumulation; FP64 eigendecomposition and per-trait algebra.
                         S_BR (the contraction of the squared rotated SNPs with D_j^-1) is
                         taken from its Chebyshev series in h^2 over the context's
                         heritabilities when the series' error bound is <= 1e-10 with at
                         most 24 terms (see gwas_sbr_info); otherwise it is contracted for
                         every pair like the other two blocks.
                         Any 0 <= p-1 <= 19 (the paper's 2 <= p <= 20, Section 3);
                         traits are processed in tiles of 32 for p-1 <= 3 (24 at
                         p-1 = 3 when S_BR comes from its series), 16 for
                         p-1 <= 10 and 8 above (the accumulators of a tile take
                         (4 + 2(p-1)) x tile + 6 x tile TMEM columns of 512, 8 x tile for
                         the C2 part of 8-trait tiles). */

/* output modes */
#define GWAS_OUT_FULL_B  0  /* double b[t][i1-i0][p]: every coefficient, SNP coefficient last */
#define GWAS_OUT_LAST_SE 1  /* float beta[t][i1-i0] followed by float se[t][i1-i0]:
                               the SNP coefficient and its standard error */

typedef struct gwas_ctx gwas_ctx;

typedef struct gwas_opts {
  int precision;      /* GWAS_FP64 or GWAS_MIXED */
  int output;         /* GWAS_OUT_FULL_B or GWAS_OUT_LAST_SE */
  int trait_block;    /* traits per internal block of gwas_solve; 0 = all traits at once */
  int device;         /* CUDA device ordinal of the context */
  int profile;        /* nonzero: time every kernel launch with CUDA events (see gwas_kernel_time) */
  size_t hbm_budget;  /* bytes the context may allocate on the device; 0 = no limit */
  void* stream;       /* cudaStream_t the context runs on; NULL = the context creates one */
  const char* tune_cache; /* JSON file of autotuned launch shapes (gwas_autotune); NULL = none.
                             gwas_setup applies the entry for its (n, p, mode, t) if present */
} gwas_opts;

/* Fill *opts with the defaults: GWAS_MIXED, GWAS_OUT_LAST_SE, trait_block 0,
 * device 0, no budget, own stream. */
GWAS_API void gwas_default_opts(gwas_opts* opts);

/*
 * gwas_setup -- create a context and perform the preloop work that involves
 * neither stream (Algorithm 5, the eigendecomposition and X'_L := Z^T X_L).
 *
 *   ctx   out: the new context (NULL on failure)
 *   n     number of individuals, 1 <= n <= 16384
 *   pm1   number of covariates p-1 (columns of X_L), 0 <= pm1 <= 19 (Section 3 states
 *         2 <= p <= 20; p = 1, no covariates, is also accepted)
 *   phi   n x n symmetric kinship matrix Phi, FP64 (only the lower triangle is read)
 *   XL    n x pm1 covariates X_L, FP64 column-major (may be NULL when pm1 == 0)
 *   t     number of traits, t >= 1
 *   h2    t heritabilities h_j^2, each in [0, 1]
 *   opts  options (NULL = defaults)
 *
 * Fails with GWAS_ERR_NOT_SPD when some h_j^2 lambda_k + 1 - h_j^2 <= 1e-12 *
 * max_k(...) (M_j not SPD; Section 3.1 needs D_j > 0), and with GWAS_ERR_ARG
 * when X_L does not have full column rank.
 */
GWAS_API int gwas_setup(gwas_ctx** ctx, int n, int pm1, const double* phi, const double* XL, int t,
               const double* h2, const gwas_opts* opts);

/*
 * gwas_load_snps -- make the genotypes X_R resident on the device and rotate
 * them by Z^T once (Algorithm 5, X'_R := Z^T X_R; Section 3.2 explains why
 * this is hoisted out of both loops).  Replaces previously loaded SNPs.
 *
 *   m   number of SNPs, m >= 1
 *   XR  n x m int8 genotypes, column-major (SNP-major), values in {0, 1, 2}
 *       (other values are accepted and used as given)
 */
GWAS_API int gwas_load_snps(gwas_ctx* ctx, int64_t m, const int8_t* XR);

/*
 * gwas_solve -- solve the grid block SNPs [i0, i1) x all t traits
 * (Algorithm 5, Y' := Z^T Y and the double loop).
 *
 *   Y    n x t phenotypes, FP64 column-major
 *   i0, i1  SNP range, 0 <= i0 <= i1 <= m
 *   out  GWAS_OUT_FULL_B: double[t][i1-i0][p];
 *        GWAS_OUT_LAST_SE: float beta[t][i1-i0], then float se[t][i1-i0].
 *
 * The standard error is sqrt(sigma^2 [S^-1]_pp) with sigma^2 = RSS/(n-p),
 * RSS the squared norm of the whitened residual (the paper defines none).
 * Returns GWAS_ERR_SINGULAR_PAIRS (a warning) when some pair's Schur
 * complement is <= 1e-10 times its diagonal entry; those outputs are NaN.
 * Where the device reads the CPU's page tables (Grace-class systems) and `out` is
 * page-locked host memory mapped for the device (cudaHostAlloc, or cudaHostRegister),
 * the kernels store the results into `out` directly, in blocks of opts.trait_block, with
 * no device staging and no copies.  (GWAS_HOST_OUTPUT=staged in the environment selects
 * the staged copies below instead.)  Any other host `out` receives the results trait
 * block by trait block through two device staging buffers, each block's copy overlapping
 * the next block's computation when `out` is page-locked (the copies reach the link's
 * full rate from memory on huge pages, e.g. cudaHostAlloc or madvise(MADV_HUGEPAGE) +
 * cudaHostRegister; registered memory on small base pages measured about half of it).
 * The staged blocks start at 1/8 of opts.trait_block traits (about 8 GB of results when
 * trait_block is 0) and grow by 1.4x per block up to it, so that the first copy
 * starts early; a device `out` is computed in blocks of opts.trait_block.
 */
GWAS_API int gwas_solve(gwas_ctx* ctx, const double* Y, int64_t i0, int64_t i1, void* out);

/*
 * gwas_solve_stream -- gwas_solve for grids whose results do not fit in host
 * memory at once (the output stream of Section 4, double-buffered).
 *
 * The traits are processed in blocks of block_traits.  The results of block b
 * (traits [j0, j0+nb)) are copied to host_buf[b % 2] on a side stream while block
 * b+1 is computed; once a copy has landed, fn(user, j0, nb, buf) is called on the
 * calling thread, and buf is reused (for block b+2) only after fn returns.  Each
 * buffer must hold one block in the output layout of the context:
 *   GWAS_OUT_FULL_B  double[nb][i1-i0][p]
 *   GWAS_OUT_LAST_SE float beta[nb][i1-i0], then float se[nb][i1-i0]
 * i.e. block_traits * (i1-i0) * (8p or 8) bytes.  Page-locked buffers let the
 * copies overlap the computation; pageable ones work but serialise the copies.
 */
typedef void (*gwas_block_fn)(void* user, int j0, int nb, const void* host_block);
GWAS_API int gwas_solve_stream(gwas_ctx* ctx, const double* Y, int64_t i0, int64_t i1, int block_traits,
                               void* host_buf0, void* host_buf1, gwas_block_fn fn, void* user);

/*
 * gwas_solve_ooc -- Algorithm 5 for genotype sets larger than device memory: the
 * out-of-core setting of Section 4, in which slabs of X_R are streamed through two
 * buffers (double buffering) while the previous slab is processed.  Here the slabs come
 * from host memory; each is uploaded on a side stream while the previous one is computed,
 * converted and rotated on the device exactly as gwas_load_snps does (the preloop of
 * Section 4.1, fused into the loop instead of written back), and solved against every
 * trait.  Results leave through the caller's two host buffers, one (slab, trait block)
 * piece at a time.
 *
 *   m, XR         SNPs and their int8 genotypes, n x m column-major (SNP i at XR + i*n),
 *                 host memory (pageable or page-locked) or device memory
 *   slab          SNPs per slab, >= 0 (0 = 2^20); rounded up to a multiple of 128
 *   Y             n x t traits, FP64 (host or device)
 *   block_traits  traits per piece, >= 1
 *   host_buf0/1   host buffers, each large enough for one piece of slab x block_traits
 *                 pairs in gwas_solve's layout (for nb traits and i1-i0 SNPs)
 *   fn            called on the calling thread for every piece, in order:
 *                 fn(user, i0, i1, j0, nb, host_block) for SNPs [i0, i1) x traits
 *                 [j0, j0+nb); host_block stays valid until fn returns
 *
 * The per-trait operands of all t traits are prepared once; each slab is uploaded,
 * converted and rotated once.  Pieces arrive slab by slab, trait blocks in order within a
 * slab.  The results equal those of gwas_load_snps(m, XR) followed by gwas_solve, bit for
 * bit.  Genotypes of an earlier gwas_load_snps are released first; the context holds none
 * afterwards.  Fails with GWAS_ERR_STATE while serving requests are pending.  Device
 * memory: the slab arrays (about 8 bytes per SNP and individual on either path), two int8
 * slabs, two output staging pieces and the operands of all traits (about 32 KB per trait
 * and 1000 individuals on the mixed path).
 */
typedef void (*gwas_slab_fn)(void* user, int64_t i0, int64_t i1, int j0, int nb, const void* host_block);
GWAS_API int gwas_solve_ooc(gwas_ctx* ctx, int64_t m, const int8_t* XR, int64_t slab, const double* Y,
                            int block_traits, void* host_buf0, void* host_buf1, gwas_slab_fn fn, void* user);

/*
 * Serving (continuous batching).  gwas_submit queues a request: tk traits Y
 * (n x tk, FP64) with their own heritabilities h2k, solved against the resident
 * SNPs [i0, i1).  A scheduler thread of the context admits queued requests while
 * their operands fit the serving arena in HBM, prepares them, and runs rounds of
 * the fused kernel over work units of every admitted request, so requests that
 * arrive while others run join the next round.  Results are the same as a
 * separate gwas_solve of the request (the mixed path).  The caller's Y and h2k
 * are copied before gwas_submit returns.  `out` (same layout as gwas_solve for
 * tk traits and i1-i0 SNPs) must be device memory or page-locked host memory and
 * must stay valid until the request has finished.  Requires GWAS_MIXED and
 * loaded genotypes.  gwas_submit, gwas_poll and gwas_wait are safe to call from
 * one host thread.
 */
GWAS_API int gwas_submit(gwas_ctx* ctx, const double* Y, int tk, const double* h2k, int64_t i0, int64_t i1, void* out,
                         uint64_t* req_id);
/* *done = 1 once the request has finished; returns its status (GWAS_OK, a warning or an error). */
GWAS_API int gwas_poll(gwas_ctx* ctx, uint64_t req_id, int* done);
/* Blocks until the request finishes or timeout_s (seconds; < 0: no limit) passes (GWAS_ERR_TIMEOUT). */
GWAS_API int gwas_wait(gwas_ctx* ctx, uint64_t req_id, double timeout_s);
/* Host steady-clock times (seconds) of a request's submission, admission and completion. */
GWAS_API int gwas_request_times(gwas_ctx* ctx, uint64_t req_id, double* t_submit, double* t_admit, double* t_done);
/* Rounds the serving loop has run since it started, and how many of them were replays of
 * the captured CUDA graph of a round (the work-list upload and the persistent kernel launch;
 * the first round launches directly and is then captured). */
GWAS_API int gwas_serve_stats(const gwas_ctx* ctx, int64_t* rounds, int64_t* graph_rounds);

/* Replace the t heritabilities given at setup (same t). */
GWAS_API int gwas_set_h2(gwas_ctx* ctx, int t, const double* h2);

/* Number of pairs flagged singular by the last gwas_solve. */
GWAS_API int64_t gwas_singular_count(const gwas_ctx* ctx);

/* How gwas_setup computed Phi = Z Lambda Z^T.  *steps >= 0: the FP32 eigensolver, refined to FP64
 * accuracy by the iteration of Ogita and Aishima (2018) with FP64-accurate products on the tensor
 * cores, took *steps refinement steps until max |(Z^T Z - I)_ij| and
 * max_{i != j} |(Z^T Phi Z)_ij| / max |lambda| were both <= 16 u sqrt(n), u = 2^-53;
 * *steps = -1: the FP64 eigensolver (cuSOLVER Dsyevd) computed it, because n > 2048, the
 * refinement did not converge within 8 steps, the FP32 solver failed, or GWAS_EIG=fp64 was set.  Either way Lambda
 * is ascending and Z column-major.  Returns GWAS_OK or GWAS_ERR_ARG (NULL argument). */
GWAS_API int gwas_eig_info(const gwas_ctx* ctx, int* steps);

/* The mixed path's e2m1 operands.  At p = 4, for blocks whose S_BR is interpolated (gwas_sbr_info)
 * and with the CTA-pair launch shape (gwas_tune_shape), the fused kernel contracts the genotypes
 * and the fixed-point slices of the per-trait columns as e2m1 values on the block-scaled FP4 tensor
 * cores (tcgen05 kind::mxf4): the genotypes are exact, each 9-bit slice digit q is split into three
 * e2m1 digits, q = 64 d0 + 8 d1 + d2 with |d| <= 4, and the three digits are contracted into the
 * slice's accumulator with scale factors 2^6, 2^3 and 2^0.  Every partial sum is the same integer as
 * with bf16 slices, so the results are identical; the kernel streams half the operand bytes.
 *   *ready     1 when the loaded genotypes have their e2m1 copy: a one-time gwas_load_snps at p = 4
 *              of genotypes that are all in {0, +-1, +-2, +-3, +-4, +-6} (not set by the slabs of
 *              gwas_solve_ooc, under GWAS_FP4=0, in a context with an HBM budget, or where the
 *              device had no room for the copy: mpad x roundup(n, 256) / 2 bytes; a block whose
 *              e2m1 trait digits find no room runs on bf16 operands)
 *   *launches  launches of the e2m1 kernel since the context was created
 * Either pointer may be NULL.  Returns GWAS_OK or GWAS_ERR_ARG (NULL context). */
GWAS_API int gwas_fp4_info(gwas_ctx* ctx, int* ready, int64_t* launches);

/* Number of kernels this context launched since it was created. */
GWAS_API int64_t gwas_kernel_launches(const gwas_ctx* ctx);

/*
 * gwas_autotune -- choose the mixed path's fused-kernel launch shape for this context by
 * timing the candidates on a sample of the grid (the loop tiles of the paper are tuned
 * empirically on the target machine, Section 5).
 *
 *   Y         traits as for gwas_solve; the first t_sample of them are used
 *   t_sample  traits of the sample (<= t; <= 0: min(t, 1024))
 *   m_sample  SNPs of the sample, from SNP 0 (<= m; <= 0: min(m, 2^17))
 *   best_ms   out (may be NULL): device time of one solve of the sample with the chosen shape
 *
 * Candidates: the one-CTA shape for every p; for p = 4 also the one-CTA shape with 8
 * epilogue warps and the CTA pair; each with 4, 8, 16, 32 or 64 SNP tiles per traversal group.  The
 * fastest is kept unless the default shape is within 2 % of it.  The context uses the choice
 * from then on, and it is written to opts.tune_cache when that was given.  Results do not
 * depend on the shape beyond rounding.  Mixed precision only (GWAS_ERR_UNSUPPORTED
 * otherwise); GWAS_ERR_STATE before gwas_load_snps or while the serving loop runs.
 */
GWAS_API int gwas_autotune(gwas_ctx* ctx, const double* Y, int t_sample, int64_t m_sample, double* best_ms);

/* The context's launch shape: shape[0..4] = cluster CTAs along SNPs, along traits,
 * epilogue warps, CTA-pair mode (0/1), SNP tiles per traversal group.
 *
 * Developer overrides, read from the environment at each launch (they take precedence over
 * the tuned shape; for measurements, not for production use):
 *   GWAS_FUSED_SHAPE="CSxCTxEPW[xPAIR]"  launch shape at p = 4: "1x1x16" (default), "1x1x8" or
 *                                         "2x1x16x1" (the CTA pair); other values are ignored
 *   GWAS_FUSED_GROUP=<k>                  SNP tiles per traversal group
 *   GWAS_SERVE_SLOTS=<k>, GWAS_SERVE_ROUND=<k>  serving arena trait-tile slots and units per round
 *   GWAS_HOST_OUTPUT=staged               gwas_solve copies page-locked host outputs through device
 *                                         staging instead of storing them from the kernels
 *   GWAS_HOST_INPUT=staged                gwas_load_snps (mixed precision) copies page-locked host
 *                                         genotypes to the device instead of reading them from the
 *                                         conversion kernel
 *   GWAS_S_BR=exact                       the mixed path contracts S_BR for every pair (read when a
 *                                         context plans it: its first solve, or after gwas_set_h2)
 *   GWAS_POOL=0                           device buffers from cudaMalloc/cudaFree instead of the
 *                                         library's pool (read once per process)
 *   GWAS_EIG=fp64                         gwas_setup computes the eigendecomposition with the FP64
 *                                         solver (see gwas_eig_info)
 *   GWAS_FP4=0                            gwas_load_snps makes no e2m1 copy of the genotypes: the
 *                                         fused kernel runs on bf16 operands (see gwas_fp4_info) */
GWAS_API int gwas_tune_shape(const gwas_ctx* ctx, int* shape);

/* Accumulated device time (ms, from CUDA events recorded on the context's stream
 * around each launch) and launch count of one kernel family since the last
 * gwas_reset_timers; zero unless the context was created with opts.profile.
 * Families: "eigendecomposition", "rotate_fp64", "prep_fp64", "fused_fp64",
 * "setup_rotation_operands", "slice_rows", "genotypes_bf16", "xgemm_rotate_snps",
 * "slice_snp_squares", "xgemm_rotate_traits", "prep_traits", "xgemm_back_rotate",
 * "pack_trait_columns", "cheb_nodes" (S_BR at the node heritabilities), "cheb_coefficients",
 * "fused"; and, inside "eigendecomposition", "eig_fp32_solver", "eig_refine_residuals" (R and S of
 * each refinement step) and "eig_refine_update". */
GWAS_API int gwas_kernel_time(const gwas_ctx* ctx, const char* kernel, double* ms, int64_t* launches);
GWAS_API void gwas_reset_timers(gwas_ctx* ctx);

/*
 * gwas_sbr_info -- how the mixed path of this context obtains S_BR = sum_k e_jk x'^2_ik, the
 * pair's diagonal entry of Algorithm 5 (the contraction (X'_R o X'_R)^T D_j^-1).
 *
 * For a SNP, S_BR is a positive combination of the functions h -> 1/(1 - h + h lambda_k) of the
 * heritability.  Its interpolant at the Chebyshev points of [lo, hi], the range of the
 * context's heritabilities, has relative error at most omega(h)/omega(h*_k) per term (omega the
 * node polynomial, h*_k = 1/(1 - lambda_k) the term's pole), taken over the eigen-directions
 * that SNPs centred against X_L reach.  When that bound is <= 1e-10 for some number of terms
 * R <= 24, the library contracts S_BR exactly at the R node heritabilities once per loaded
 * genotype set, converts the node values to Chebyshev coefficients (FP64) and the fused kernel
 * evaluates the series per pair; its K loop then streams only the other two blocks' operands.
 * Otherwise (e.g. an eigenvalue near 0 reached by the SNPs with heritabilities near 1), and
 * under GWAS_S_BR=exact, S_BR is contracted for every pair.  Serving requests (their own
 * heritabilities) and single-trait blocks always contract it.
 *
 *   terms  out: R, or 0 when S_BR is contracted per pair (and for GWAS_FP64 contexts)
 *   lo, hi out: the interpolation interval;  bound  out: the relative error bound
 * The plan is made (if not yet) for the current heritabilities; call after gwas_load_snps or a
 * gwas_solve for a mixed context.
 */
GWAS_API int gwas_sbr_info(gwas_ctx* ctx, int* terms, double* lo, double* hi, double* bound);

/*
 * gwas_cheb_plan -- the planning rule of gwas_sbr_info on its own (host only, no device work):
 * the least R in [4, 24] whose bound (above) is <= tol for the eigenvalues lam[k] with
 * reach[k] != 0 on [lo, hi] (0 <= lo < hi <= 1), or *R = 0 when none is; *bound (may be NULL)
 * receives the bound of the last R tried.  GWAS_ERR_ARG on invalid arguments.
 */
GWAS_API int gwas_cheb_plan(int n, const double* lam, const unsigned char* reach, double lo, double hi, double tol,
                            int* R, double* bound);

/*
 * gwas_solve_fp64_noalloc -- the FP64 per-trait preparation and the fused FP64
 * contraction + solve of gwas_solve, for callers that cannot allocate device
 * memory.  The paper has no counterpart: it serves host applications whose
 * memory manager owns the whole device (a framework's caching allocator, an
 * arena fixed at start-up) and plug-in code that is handed only buffers and a
 * stream.  It calls no cudaMalloc, cudaFree or allocating library routine; its
 * scratch is a fixed 8 MiB device array inside the library, which every GPU
 * that loads the library keeps until the process exits.
 *
 * Inputs are already rotated by the eigenvectors Z of Phi = Z diag(lam) Z^T.
 * Every array must be device memory of the current device (or managed memory);
 * anything else (a host pointer, pinned or not, or another device's memory) is
 * refused with GWAS_ERR_ARG before any device work:
 *   lam  n eigenvalues of Phi          XLt  [pm1][n] rows Z^T x_L,l
 *   Xt   [m][n] rows Z^T x_i (FP64)    Yt   [t][n] rows Z^T y_j
 *   h2   t heritabilities, each in [0, 1]
 * out: GWAS_OUT_FULL_B double[t][m][p]; GWAS_OUT_LAST_SE float beta[t][m], then
 * float se[t][m].  stream: cudaStream_t (NULL = legacy default stream); the call
 * returns after the stream has finished.  *singular (may be NULL) receives the
 * number of singular pairs.
 *
 * The scratch must hold t (p+1) n + t (pm1^2 + pm1 + 1) doubles plus 256 bytes:
 * larger requests return GWAS_ERR_UNSUPPORTED before any device work.  The
 * array's device address is looked up on every call with the current device, so
 * a context torn down and created again (cudaDeviceReset) is handled.  The
 * heritabilities are checked on the device before any result is written: h2
 * outside [0, 1] returns GWAS_ERR_ARG, and a D_j = h2 lam + 1 - h2 with an entry
 * <= 1e-12 of its largest returns GWAS_ERR_NOT_SPD (the check gwas_setup makes).
 * Every call shares the one array and it keeps the last call's contents: calls
 * that overlap on the GPU race on it.  Returns GWAS_OK, GWAS_ERR_SINGULAR_PAIRS
 * (a warning), GWAS_ERR_ARG, GWAS_ERR_NOT_SPD, GWAS_ERR_UNSUPPORTED or
 * GWAS_ERR_CUDA; gwas_last_error is not set.
 */
GWAS_API int gwas_solve_fp64_noalloc(int n, int pm1, const double* lam, const double* XLt, const double* Xt,
                                     int64_t m, const double* Yt, const double* h2, int t, int output, void* out,
                                     void* stream, int64_t* singular);

/*
 * Self-test of failure detection: launches one kernel that waits on a barrier that
 * nothing completes, with the same bounded-wait code every kernel of the library
 * uses but a limit of limit_s seconds (0 < limit_s <= 10).  Returns GWAS_ERR_TIMEOUT
 * (the expected outcome: the wait gave up and reported it) with *waited_s the time it
 * waited, GWAS_OK if the barrier completed, or GWAS_ERR_CUDA.  The device stays usable.
 */
GWAS_API int gwas_check_bounded_wait(int device, double limit_s, double* waited_s);

/*
 * Self-test of the fused kernel's epilogue arithmetic: evaluates on the device, for each of the
 * count values x[i] (host array, 1 <= count <= 2^20), the reciprocal and the square root that
 * the mixed path's per-pair solve uses (the hardware approximation of 1/x refined by one
 * Newton-Raphson step, and the hardware approximation of sqrt(x)) beside CUDA's correctly
 * rounded __frcp_rn and __fsqrt_rn.  out (host, 4 * count floats) receives, per value, those
 * four results in that order.  Returns GWAS_OK, GWAS_ERR_ARG or GWAS_ERR_CUDA.
 */
GWAS_API int gwas_check_epilogue_math(int device, const float* x, int count, float* out);

/* One-line description of the last failure on ctx (or of the last failed
 * gwas_setup when ctx is NULL).  Owned by the library. */
GWAS_API const char* gwas_last_error(const gwas_ctx* ctx);

/* Free every device and host resource of the context; its device buffers go back to the
 * library's device memory pool (below).  NULL is ignored. */
GWAS_API void gwas_destroy(gwas_ctx* ctx);

/*
 * Device memory pool.  Every context's device buffers come from one stream-ordered pool
 * per device that the library keeps for the life of the process, and memory a context
 * gives back stays reserved in it for the next context: a step that sets up, solves and
 * destroys a context does not map and unmap its buffers again (at n = 1000, m = 10^6 that
 * is ~10 GB, ~6 ms per step).  A buffer is usable from any stream once the call that made
 * it returns, and is handed out again only after all work on the device has completed.
 *
 * gwas_pool_info: *reserved = bytes the pool holds from the device, *used = bytes in live
 *   context buffers (either pointer may be NULL); both 0 while the pool is not in use
 *   (GWAS_POOL=0, or no context has allocated on the device yet).
 * gwas_pool_trim: gives reserved memory that no live buffer uses back to the device, until
 *   at most keep_bytes stay reserved (0: everything unused).
 * Both return GWAS_OK, GWAS_ERR_ARG (no such device, or a negative device) or GWAS_ERR_CUDA;
 * gwas_last_error is not set.  Thread-safe.
 */
GWAS_API int gwas_pool_info(int device, uint64_t* reserved, uint64_t* used);
GWAS_API int gwas_pool_trim(int device, uint64_t keep_bytes);

#ifdef __cplusplus
}
#endif
#endif /* GWAS_GB300_H */
