// Launch of the single-trait kernel (gemv_impl.cuh) for 0 <= p - 1 <= 7; 8 <= p - 1 <= 19
// is instantiated in gemv_wide.cu.
#include "gemv_impl.cuh"

bool gemv1_supported(int q, int Kpad) { return q >= 0 && q <= MIXED_MAX_Q && Kpad % GK == 0; }

int launch_gemv1(gwas_ctx* c, int q, const FusedArgs& a, const __nv_bfloat16* G, const __nv_bfloat16* A2,
                 const __nv_bfloat16* B1, const __nv_bfloat16* B2) {
  if (a.nsnp <= 0) return GWAS_OK;
  if (!gemv1_supported(q, a.Kpad)) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "single-trait kernel: p-1 out of range");
  const int TT = mixed_tt(q);
  CUtensorMap mg, ma, m1, m2;
  if (!make_bf16_map(&mg, G, a.mpad, a.Kpad, 128, GK) || !make_bf16_map(&ma, A2, 3ull * a.mpad, a.Kpad, 128, GK) ||
      !make_bf16_map_strided(&m1, B1, c1_groups(q), a.Kpad, (uint64_t)TT * a.Kpad, c1_groups(q), GK) ||
      !make_bf16_map_strided(&m2, B2, 4, a.Kpad, (uint64_t)TT * a.Kpad, 4, GK))
    return ctx_fail(c, GWAS_ERR_CUDA, "tensor map encoding failed");
  if (q > 7) return launch_gemv1_wide(c, q, a, mg, ma, m1, m2);
  Q_DISPATCH(q, return launch_gemv1_q<Q>(c, a, mg, ma, m1, m2));
  return GWAS_OK;
}
