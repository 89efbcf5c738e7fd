// FP32-arithmetic diffusion with the geometric factors recomputed from the trilinear element map
// at every application (FP64 L-vectors in and out).
#include "apply_kernel.cuh"

namespace ceedgb {
int launch_apply_qf32geo(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  if (((uintptr_t)r.qdata & 15) != 0) return fail(CEED_ERR_INVALID, "qdata must be 16-byte aligned");
  const bool colloc = (m->Q == m->P);
#define CEEDGB_CASE(PP)                                                                 \
  case PP:                                                                             \
    return colloc ? launch_colours<PP, PP, OP_DIFF_GEO, float, float>(m, m->tab32, r, s) \
                  : launch_colours<PP, PP + 1, OP_DIFF_GEO, float, float>(m, m->tab32, r, s);
  switch (m->P) {
    CEEDGB_CASE(2)
    CEEDGB_CASE(3)
    CEEDGB_CASE(4)
    CEEDGB_CASE(5)
    CEEDGB_CASE(6)
    CEEDGB_CASE(7)
    CEEDGB_CASE(8)
    CEEDGB_CASE(9)
    default:
      return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
  }
#undef CEEDGB_CASE
}
}  // namespace ceedgb
