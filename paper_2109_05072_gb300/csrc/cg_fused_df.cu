// Fused PCG iteration with the FP64-accurate double-float operator (GLL collocated diffusion).
#include "cg_fused.cuh"

namespace ceedgb {
int launch_cg_fused_df(ceed_mesh_t m, const CgFusedArgs &g, int ne, cudaStream_t s, unsigned *grid) {
  return dispatch_cg_fused<CEED_OP_DIFFUSION, DF, DF>(m->P, g, m->tabdf, ne, s, grid);
}
}  // namespace ceedgb
