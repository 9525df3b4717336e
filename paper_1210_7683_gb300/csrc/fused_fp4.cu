// Launch of the fused kernel's CTA-pair shape with S_BR interpolated on e2m1 operands
// (fused_impl.cuh, FP4), in a translation unit of its own so that the library's sources compile
// in parallel.
#include "fused_impl.cuh"

int launch_fused_cheb_pair_fp4(gwas_ctx* c, const FusedArgs& a, const uint8_t* G4, const uint8_t* B1_4, int b_tiles) {
  if (a.cheb_R < 2 || a.cheb_R > CHEB_MAX_R) return ctx_fail(c, GWAS_ERR_ARG, "Chebyshev terms outside [2, 24]");
  if (a.Kp4 <= 0 || a.Kp4 % BK4) return ctx_fail(c, GWAS_ERR_ARG, "e2m1 operands: K not a multiple of 256");
  // boxes of 128 bytes (256 e2m1 values) x 128 genotype rows, or x 120 rows of one digit of the
  // CTA's half of a trait tile's C1 columns; the second map: a tile's Chebyshev coefficient rows
  // 0..CHEB_MAX_R, for the epilogue's staging
  CUtensorMap mg, m1, mc;
  if (!make_u8_map(&mg, G4, a.mpad, a.Kp4 / 2, BM) ||
      !make_u8_map(&m1, B1_4, (uint64_t)b_tiles * FP4_TILE_ROWS, a.Kp4 / 2, F4_HALF) ||
      !make_f32_map(&mc, a.cheb_coef, CHEB_MAX_R + 1, a.cheb_ld, CHEB_MAX_R + 1, BM))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  c->fp4_launches++;
  return launch_shape<epw_interp(3), false, true, 3, true, true>(c, a, mg, mc, m1, m1);
}
