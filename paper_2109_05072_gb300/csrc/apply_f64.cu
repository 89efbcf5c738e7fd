// FP64 operator: FP64 quadrature data, FP64 contractions.
#include "apply_kernel.cuh"

namespace ceedgb {
int launch_apply_f64(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  return dispatch_apply<double, double>(m, m->tab64, r, s);
}
}  // namespace ceedgb
