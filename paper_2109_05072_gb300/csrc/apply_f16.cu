// FP32-arithmetic operator with f16 quadrature data (FP64 L-vectors in and out).
#include "apply_kernel.cuh"

namespace ceedgb {
int launch_apply_qf16(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  return dispatch_apply<float, __half>(m, m->tab32, r, s);
}
}  // namespace ceedgb
