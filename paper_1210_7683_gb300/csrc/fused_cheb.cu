// Launches of the fused contraction + Schur solve kernel with S_BR evaluated from its
// Chebyshev series in h^2 (fused_impl.cuh, INTERP) for 0 <= p - 1 <= 7, in a translation
// unit of its own so that the library's sources compile in parallel.
#include "fused_impl.cuh"

int launch_fused_cheb(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* B1,
                      int b_tiles) {
  if (q < 0 || q > 7) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "interpolated fused kernel: p-1 outside [0, 7]");
  if (a.cheb_R < 2 || a.cheb_R > CHEB_MAX_R) return ctx_fail(c, GWAS_ERR_ARG, "Chebyshev terms outside [2, 24]");
  // the x'^2 planes and the C2 trait rows are not read: their maps describe the C1 operands
  CUtensorMap mg, m1;
  const int r1 = c1_rows_of(q, true), b1box = r1 <= 256 ? r1 : r1 / 2;
  if (!make_bf16_map(&mg, G, a.mpad, a.Kpad, BM, BK) ||
      !make_bf16_map(&m1, B1, (uint64_t)b_tiles * r1, a.Kpad, b1box, BK))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  // q = 3: 24-trait tiles, 12 epilogue warps of 8 traits
  Q_DISPATCH(q, return launch_shape<epw_interp(Q), false, false, Q, true>(c, a, mg, mg, m1, m1));
  return GWAS_OK;
}

int launch_fused_cheb_pair(gwas_ctx* c, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* B1,
                           int b_tiles) {
  if (a.cheb_R < 2 || a.cheb_R > CHEB_MAX_R) return ctx_fail(c, GWAS_ERR_ARG, "Chebyshev terms outside [2, 24]");
  // each CTA of the pair: its own 128 SNP rows and its half (120 rows) of the tile's 240 C1 rows;
  // the second map: a tile's Chebyshev coefficient rows 0..CHEB_MAX_R, for the epilogue's staging
  CUtensorMap mg, m1, mc;
  if (!make_bf16_map(&mg, G, a.mpad, a.Kpad, BM, BK) ||
      !make_bf16_map(&m1, B1, (uint64_t)b_tiles * c1_rows_of(3, true), a.Kpad, c1_rows_of(3, true) / 2, BK) ||
      !make_f32_map(&mc, a.cheb_coef, CHEB_MAX_R + 1, a.cheb_ld, CHEB_MAX_R + 1, BM))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  return launch_shape<epw_interp(3), false, true, 3, true>(c, a, mg, mc, m1, m1);
}
