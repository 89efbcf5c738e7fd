// FP64-accurate mass operator on the FP32 pipe: double-float interpolation by compensated even-odd
// contractions and a double-float pointwise product (own translation unit: compiles in parallel
// with the diffusion instantiations).
#include "apply_kernel.cuh"

namespace ceedgb {
int launch_apply_df_mass(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  return dispatch_apply_op<CEED_OP_MASS, DF, DF>(m, m->tabdf, r, s);
}
}  // namespace ceedgb
