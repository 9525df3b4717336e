// Launches of the fused kernel with S_BR evaluated from its Chebyshev series in h^2
// (fused_impl.cuh, INTERP) for 8 <= p - 1 <= 19: 16-trait tiles up to p - 1 = 10 and 8-trait
// tiles above, in a translation unit of their own.
#include "fused_impl.cuh"

int launch_fused_cheb_wide(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* B1,
                           int b_tiles) {
  if (q < 8 || q > MIXED_MAX_Q) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "interpolated fused kernel: p-1 outside [8, 19]");
  if (a.cheb_R < 2 || a.cheb_R > CHEB_MAX_R) return ctx_fail(c, GWAS_ERR_ARG, "Chebyshev terms outside [2, 24]");
  CUtensorMap mg, m1;
  const int r1 = c1_rows_of(q, true), b1box = r1 <= 256 ? r1 : r1 / 2;
  if (!make_bf16_map(&mg, G, a.mpad, a.Kpad, BM, BK) ||
      !make_bf16_map(&m1, B1, (uint64_t)b_tiles * r1, a.Kpad, b1box, BK))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  Q_DISPATCH_WIDE(q, return launch_shape<epw_interp(Q), false, false, Q, true>(c, a, mg, mg, m1, m1));
  return GWAS_OK;
}
