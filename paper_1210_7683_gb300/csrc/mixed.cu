// Mixed-precision path (tensor cores).  Placeholder until the tcgen05 kernels land.
#include "gwas_internal.cuh"

int mixed_load(gwas_ctx* c, const int8_t*) { return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "mixed path not built"); }
int mixed_solve_block(gwas_ctx* c, const double*, int, int, int64_t, int64_t, int64_t, void*) {
  return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "mixed path not built");
}
void mixed_free(gwas_ctx*) {}
