// Tensor-core (tcgen05, kind::tf32) kernels of the PUFE hot path.
#include "pufe_internal.h"

namespace pufe {

pufe_status launch_assemble_tc(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                               cudaStream_t s) {
  (void)ctx; (void)V; (void)what; (void)H; (void)S; (void)s;
  return fail(PUFE_EINVAL, "PUFE_TF32X3 assembly is not available in this build");
}

pufe_status launch_density_tc(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f,
                              int nocc, double *rho, cudaStream_t s) {
  (void)ctx; (void)C; (void)ldc; (void)f; (void)nocc; (void)rho; (void)s;
  return fail(PUFE_EINVAL, "PUFE_TF32X3 density is not available in this build");
}

}  // namespace pufe
