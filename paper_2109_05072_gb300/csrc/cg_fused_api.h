// Launchers of the fused persistent PCG iteration, one translation unit per operator precision
// (they compile in parallel): cg_fused_f64.cu, cg_fused_f32.cu (F32, BF16 and on-the-fly-geometry
// quadrature data), cg_fused_df.cu (double-float).
#pragma once

#include "internal.h"

namespace ceedgb {

constexpr int CGF_MAX_COLORS = 64;
constexpr int CGF_MAX_GRID = 8192;     // resident blocks of a fused launch (partials per reduction)

struct CgFusedArgs;

int launch_cg_fused_f64(ceed_mesh_t m, const CgFusedArgs &g, int ne, cudaStream_t s, unsigned *grid);
int launch_cg_fused_f32(ceed_mesh_t m, int prec, const CgFusedArgs &g, int ne, cudaStream_t s, unsigned *grid);
int launch_cg_fused_df(ceed_mesh_t m, const CgFusedArgs &g, int ne, cudaStream_t s, unsigned *grid);

}  // namespace ceedgb
