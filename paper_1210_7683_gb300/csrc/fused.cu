// Launches of the fused contraction + Schur solve kernel (fused_impl.cuh) for 0 <= p - 1 <= 7,
// with the optional 8-epilogue-warp and CTA-pair shapes of p = 4; 8 <= p - 1 <= 19 is
// instantiated in fused_wide.cu.
#include "fused_impl.cuh"

namespace {

struct Shape {
  int cs, ct, epw, pair;
};

// The context's kernel shape (autotuned or default).  Shapes other than 1x1x16 exist for q = 3
// only (1x1x8 and the CTA pair 2x1x16x1); every other q runs 1x1x16.
// GWAS_FUSED_SHAPE="CSxCTxEPW[xPAIR]" overrides it (q = 3) when it names one of those shapes.
Shape shape_of(const gwas_ctx* c, int q) {
  Shape sh{1, 1, 16, 0};
  if (q != 3) return sh;
  if (c) sh = {c->tune.cs, c->tune.ct, c->tune.epw, c->tune.pair};
  if (const char* e = getenv("GWAS_FUSED_SHAPE")) {
    int cs = 0, ct = 0, epw = 0, pr = 0;
    const int k = sscanf(e, "%dx%dx%dx%d", &cs, &ct, &epw, &pr);
    if (k >= 3 && fused_shape_supported(q, cs, ct, epw, k == 4 ? pr : 0)) sh = {cs, ct, epw, k == 4 ? pr : 0};
  }
  return sh;
}

}  // namespace

int fused_trait_tile_multiple() { return 4; }

int fused_pair_layout(const gwas_ctx* c, int q) { return shape_of(c, q).pair; }

bool fused_shape_supported(int q, int cs, int ct, int epw, int pair) {
  if (cs == 1 && ct == 1 && epw == 16 && !pair) return true;
  if (q != 3) return false;
  if (cs == 1 && ct == 1 && epw == 8 && !pair) return true;
  return cs == 2 && ct == 1 && epw == 16 && pair == 1;
}

int launch_fused(gwas_ctx* c, int q, const FusedArgs& args, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2) {
  FusedArgs a = args;
  if (a.n_stiles == 0 || a.n_ttiles == 0) return GWAS_OK;
  if (q < 0 || q > MIXED_MAX_Q) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "fused kernel: p-1 outside [0, 19]");
  // S_BR from its Chebyshev series: the C1 operands only, in the one-CTA shape or the CTA pair
  if (a.cheb_coef) {
    const int bt = (a.n_ttiles + 3) / 4 * 4;
    if (q == 3 && shape_of(c, q).pair) return launch_fused_cheb_pair(c, a, G, B1, bt);
    return q > 7 ? launch_fused_cheb_wide(c, q, a, G, B1, bt) : launch_fused_cheb(c, q, a, G, B1, bt);
  }
  if (q > 7) return launch_fused_wide(c, q, a, G, A2, B1, B2, false, (a.n_ttiles + 3) / 4 * 4);
  // the node sums of the interpolated S_BR use the one-CTA operand layout
  const Shape sh = a.full_b == 2 ? Shape{1, 1, 16, 0} : shape_of(c, q);
  const int ttiles_pad = (a.n_ttiles + 3) / 4 * 4;   // trait operands are allocated for a multiple of 4 tiles
  CUtensorMap mg, ma, m1, m2;
  bool maps_ok;
  if (sh.pair)  // boxes of 128 SNP rows, 160 C1 and 96 C2 trait rows (one CTA's half)
    maps_ok = make_bf16_map(&mg, G, a.mpad, a.Kpad, BM, BK) && make_bf16_map(&ma, A2, 3ull * a.mpad, a.Kpad, BM, BK) &&
              make_bf16_map(&m1, B1, (uint64_t)ttiles_pad * c1_rows(3), a.Kpad, PC1_ROWS, BK) &&
              make_bf16_map(&m2, B2, (uint64_t)ttiles_pad * c2_alloc(3), a.Kpad, PC2_ROWS, BK);
  else
    maps_ok = make_big_maps(q, &mg, &ma, &m1, &m2, a, G, A2, B1, B2, ttiles_pad);
  if (!maps_ok) return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  if (sh.pair) return launch_shape<16, false, true, 3>(c, a, mg, ma, m1, m2);
  // 8 epilogue warps of 16 traits each (q = 3): fewer warps beside the MMA issuer
  if (sh.epw == 8) return launch_shape<8, false, false, 3>(c, a, mg, ma, m1, m2);
  Q_DISPATCH(q, return launch_shape<16, false, false, Q>(c, a, mg, ma, m1, m2));
  return GWAS_OK;
}

int launch_fused_serve(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                       const __nv_bfloat16* B1, const __nv_bfloat16* B2, int b_tiles) {
  if (a.nunits == 0) return GWAS_OK;
  if (q < 0 || q > MIXED_MAX_Q) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "fused kernel: p-1 outside [0, 19]");
  if (q > 7) return launch_fused_wide(c, q, a, G, A2, B1, B2, true, b_tiles);
  CUtensorMap mg, ma, m1, m2;
  if (!make_big_maps(q, &mg, &ma, &m1, &m2, a, G, A2, B1, B2, b_tiles))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  Q_DISPATCH(q, return launch_shape<16, true, false, Q>(c, a, mg, ma, m1, m2));
  return GWAS_OK;
}
