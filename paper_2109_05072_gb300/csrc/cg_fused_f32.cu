// Fused PCG iteration with the FP32-arithmetic operators (GLL collocated diffusion, p = 1..8):
// FP32 or BF16 quadrature data, or the geometric factors rebuilt from the trilinear map (F32_GEO).
#include <cuda_bf16.h>

#include "cg_fused.cuh"

namespace ceedgb {
int launch_cg_fused_f32(ceed_mesh_t m, int prec, const CgFusedArgs &g, int ne, cudaStream_t s, unsigned *grid) {
  switch (prec) {
    case CEED_F32: return dispatch_cg_fused<CEED_OP_DIFFUSION, float, float>(m->P, g, m->tab32, ne, s, grid);
    case CEED_BF16: return dispatch_cg_fused<CEED_OP_DIFFUSION, float, __nv_bfloat16>(m->P, g, m->tab32, ne, s, grid);
    case CEED_F32_GEO: return dispatch_cg_fused<OP_DIFF_GEO, float, float>(m->P, g, m->tab32, ne, s, grid);
    default: return fail(CEED_ERR_UNSUPPORTED, "no fused CG iteration for this precision");
  }
}
}  // namespace ceedgb
