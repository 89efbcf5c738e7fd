// Batched persistent apply, FP64-accurate double-float operator (mass or diffusion).
#include "batch.cuh"

namespace ceedgb {
int launch_batch_df(int op, int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, unsigned *sync, int *err,
                    const BatchLaunch &L, cudaStream_t s, unsigned *grid) {
  const OpTab<DF> *tabs[BATCH_MAX];
  for (int k = 0; k < n; ++k) tabs[k] = &meshes[k]->tabdf;
  if (op == CEED_OP_MASS) return launch_batch<CEED_OP_MASS, DF, DF>(n, meshes, reqs, tabs, sync, err, L, s, grid);
  return launch_batch<CEED_OP_DIFFUSION, DF, DF>(n, meshes, reqs, tabs, sync, err, L, s, grid);
}
}  // namespace ceedgb
