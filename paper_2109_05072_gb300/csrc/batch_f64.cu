// Batched persistent apply, FP64 operator (mass or diffusion).
#include "batch.cuh"

namespace ceedgb {
int launch_batch_f64(int op, int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, unsigned *sync, int *err,
                     const BatchLaunch &L, cudaStream_t s, unsigned *grid) {
  const OpTab<double> *tabs[BATCH_MAX];
  for (int k = 0; k < n; ++k) tabs[k] = &meshes[k]->tab64;
  if (op == CEED_OP_MASS) return launch_batch<CEED_OP_MASS, double, double>(n, meshes, reqs, tabs, sync, err, L, s, grid);
  return launch_batch<CEED_OP_DIFFUSION, double, double>(n, meshes, reqs, tabs, sync, err, L, s, grid);
}
}  // namespace ceedgb
