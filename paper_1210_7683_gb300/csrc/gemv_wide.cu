// Launch of the single-trait kernel (gemv_impl.cuh) for 8 <= p - 1 <= 19, in a translation
// unit of its own so that the library's sources compile in parallel.
#include "gemv_impl.cuh"

int launch_gemv1_wide(gwas_ctx* c, int q, const FusedArgs& a, const CUtensorMap& mg, const CUtensorMap& ma,
                      const CUtensorMap& m1, const CUtensorMap& m2) {
  if (q < 8 || q > MIXED_MAX_Q) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "single-trait kernel: p-1 outside [8, 19]");
  Q_DISPATCH_WIDE(q, return launch_gemv1_q<Q>(c, a, mg, ma, m1, m2));
  return GWAS_OK;
}
