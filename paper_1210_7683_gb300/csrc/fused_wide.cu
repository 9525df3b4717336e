// Launches of the fused contraction + Schur solve kernel (fused_impl.cuh) for
// 8 <= p - 1 <= 19 covariates (the upper end of the paper's 2 <= p <= 20): 16-trait tiles up
// to p - 1 = 10 and 8-trait tiles above, one CTA per tile, in a translation unit of their own
// so that the library's sources compile in parallel.
#include "fused_impl.cuh"

int launch_fused_wide(gwas_ctx* c, int q, const FusedArgs& args, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                      const __nv_bfloat16* B1, const __nv_bfloat16* B2, bool serve, int b_tiles) {
  if (q < 8 || q > MIXED_MAX_Q) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "wide fused kernel: p-1 outside [8, 19]");
  const FusedArgs& a = args;
  CUtensorMap mg, ma, m1, m2;
  if (!make_big_maps(q, &mg, &ma, &m1, &m2, a, G, A2, B1, B2, b_tiles))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  if (serve) {
    Q_DISPATCH_WIDE(q, return launch_shape<epw_for(Q), true, false, Q>(c, a, mg, ma, m1, m2));
  } else {
    Q_DISPATCH_WIDE(q, return launch_shape<epw_for(Q), false, false, Q>(c, a, mg, ma, m1, m2));
  }
  return GWAS_OK;
}
