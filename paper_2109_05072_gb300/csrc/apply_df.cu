// FP64-accurate diffusion computed on the FP32 pipe: double-float values and quadrature data,
// compensated (Dot2) contractions; GLL-collocated and Gauss (q = p + 2) quadrature.
#include "apply_kernel.cuh"

namespace ceedgb {
int launch_apply_df_mass(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);

int launch_apply_df(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  if (r.op == CEED_OP_MASS) return launch_apply_df_mass(m, r, s);
  return dispatch_apply_op<CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
}
}  // namespace ceedgb
