// Batched persistent apply, FP32-arithmetic diffusion with FP32 quadrature data.
#include "batch.cuh"

namespace ceedgb {
int launch_batch_f32(int op, int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, unsigned *sync, int *err,
                     const BatchLaunch &L, cudaStream_t s, unsigned *grid) {
  if (op != CEED_OP_DIFFUSION) return fail(CEED_ERR_UNSUPPORTED, "FP32 batches support diffusion");
  const OpTab<float> *tabs[BATCH_MAX];
  for (int k = 0; k < n; ++k) tabs[k] = &meshes[k]->tab32;
  return launch_batch<CEED_OP_DIFFUSION, float, float>(n, meshes, reqs, tabs, sync, err, L, s, grid);
}
}  // namespace ceedgb
