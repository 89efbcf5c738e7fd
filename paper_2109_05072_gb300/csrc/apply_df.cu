// FP64-accurate diffusion computed on the FP32 pipe: double-float values and quadrature data,
// compensated (Dot2) contractions; GLL-collocated diffusion only.
#include "apply_kernel.cuh"

namespace ceedgb {
int launch_apply_df(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  if (((uintptr_t)r.qdata & 15) != 0) return fail(CEED_ERR_INVALID, "qdata must be 16-byte aligned");
  if (r.op != CEED_OP_DIFFUSION || m->Q != m->P)
    return fail(CEED_ERR_UNSUPPORTED, "the double-float operator covers GLL-collocated diffusion");
  switch (m->P) {
    case 2: return launch_colours<2, 2, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 3: return launch_colours<3, 3, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 4: return launch_colours<4, 4, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 5: return launch_colours<5, 5, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 6: return launch_colours<6, 6, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 7: return launch_colours<7, 7, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 8: return launch_colours<8, 8, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    case 9: return launch_colours<9, 9, CEED_OP_DIFFUSION, DF, DF>(m, m->tabdf, r, s);
    default: return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
  }
}
}  // namespace ceedgb
