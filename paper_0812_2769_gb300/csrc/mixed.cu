// Mixed precision: FP32 inner Krylov solves inside FP64 iterative refinement.
#include "internal.hpp"

gsk_status gmres_solve_mixed(gsk_ctx* ctx, const gsk_csr*, const void*, void*, int, double, const gsk_opts*,
                             gsk_info*, void*) {
  return ctx->fail(GSK_ERR_ARG, "mixed precision GMRES is not available yet");
}
gsk_status bicgstab_solve_mixed(gsk_ctx* ctx, const gsk_csr*, const void*, void*, double, const gsk_opts*,
                                gsk_info*, void*) {
  return ctx->fail(GSK_ERR_ARG, "mixed precision Bi-CGSTAB is not available yet");
}
