// Fused PCG iteration with the FP64 operator (GLL collocated diffusion, p = 1..8).
#include "cg_fused.cuh"

namespace ceedgb {
int launch_cg_fused_f64(ceed_mesh_t m, const CgFusedArgs &g, int ne, cudaStream_t s, unsigned *grid) {
  return dispatch_cg_fused<CEED_OP_DIFFUSION, double, double>(m->P, g, m->tab64, ne, s, grid);
}
}  // namespace ceedgb
