// Batch object: several meshes applied by one persistent launch, replayed through a CUDA graph.
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace ceedgb {
int launch_batch_f64(int op, int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, unsigned *sync, int *err,
                     const BatchLaunch &L, cudaStream_t s, unsigned *grid);
int launch_batch_f32(int op, int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, unsigned *sync, int *err,
                     const BatchLaunch &L, cudaStream_t s, unsigned *grid);
int launch_batch_df(int op, int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, unsigned *sync, int *err,
                    const BatchLaunch &L, cudaStream_t s, unsigned *grid);
}  // namespace ceedgb

using namespace ceedgb;

struct ceed_batch_s {
  int n = 0, op = 0, prec = 0;
  ceed_mesh_t meshes[4] = {};
  ApplyReq reqs[4];
  BatchLaunch L{256, 1, 0};
  unsigned grid = 0;
  unsigned *d_sync = nullptr;
  int *d_err = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static int batch_launch_direct(ceed_batch_s *b, cudaStream_t s) {
  if (b->prec == CEED_F64) return launch_batch_f64(b->op, b->n, b->meshes, b->reqs, b->d_sync, b->d_err, b->L, s, &b->grid);
  if (b->prec == CEED_F64_DF)
    return launch_batch_df(b->op, b->n, b->meshes, b->reqs, b->d_sync, b->d_err, b->L, s, &b->grid);
  return launch_batch_f32(b->op, b->n, b->meshes, b->reqs, b->d_sync, b->d_err, b->L, s, &b->grid);
}

static void drop_graph(ceed_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Capture one persistent launch into a graph on a private stream.
static int build_graph(ceed_batch_s *b) {
  drop_graph(b);
  cudaStream_t cs;
  CEED_CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int st = batch_launch_direct(b, cs);  // sets kernel attributes outside the capture
  if (st == CEED_OK) {
    CEED_CUDA_CHECK(cudaStreamSynchronize(cs));
    CEED_CUDA_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    st = batch_launch_direct(b, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st == CEED_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
    if (st == CEED_OK) {
      b->graph = g;
      const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
      if (ei != cudaSuccess) st = cuda_fail(ei, "cudaGraphInstantiate");
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  return st;
}

extern "C" int ceed_batch_create(int n, const ceed_mesh_t *meshes, const void *const *qdata, int prec, int op,
                                 const double *const *x, double *const *y, int nrhs, ceed_batch_t *out) {
  if (!out || !meshes || !qdata || !x || !y) return fail(CEED_ERR_INVALID, "null batch argument");
  *out = nullptr;
  if (n < 1 || n > 4) return fail(CEED_ERR_INVALID, "a batch holds 1..4 meshes");
  if (nrhs < 1) return fail(CEED_ERR_INVALID, "nrhs must be >= 1");
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  if (prec != CEED_F64 && prec != CEED_F64_DF && !(prec == CEED_F32 && op == CEED_OP_DIFFUSION))
    return fail(CEED_ERR_UNSUPPORTED, "batches support FP64 and double-float mass/diffusion, and FP32 diffusion");
  ceed_batch_s *b = new (std::nothrow) ceed_batch_s();
  if (!b) return fail(CEED_ERR_OOM, "host allocation");
  b->n = n;
  b->op = op;
  b->prec = prec;
  for (int k = 0; k < n; ++k) {
    if (!meshes[k] || !qdata[k] || !x[k] || !y[k] || x[k] == y[k]) {
      delete b;
      return fail(CEED_ERR_INVALID, "bad mesh, qdata or vector in the batch");
    }
    if (((uintptr_t)qdata[k] & 15) != 0) {
      delete b;
      return fail(CEED_ERR_INVALID, "qdata must be 16-byte aligned");
    }
    b->meshes[k] = meshes[k];
    ApplyReq &r = b->reqs[k];
    r.op = op;
    r.prec = prec;
    r.qdata = qdata[k];
    r.x = x[k];
    r.y = y[k];
    r.ncol = meshes[k]->ncomp * nrhs;
    r.masked = 0;
  }
  cudaError_t e = cudaMalloc(&b->d_sync, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_sync, 0, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(b->d_sync);
    cudaFree(b->d_err);
    delete b;
    return cuda_fail(e, "batch device state");
  }
  if (int st = build_graph(b)) {
    drop_graph(b);
    cudaFree(b->d_sync);
    cudaFree(b->d_err);
    delete b;
    return st;
  }
  *out = b;
  return CEED_OK;
}

extern "C" int ceed_batch_apply(ceed_batch_t b, void *stream) {
  if (!b) return fail(CEED_ERR_INVALID, "null batch");
  if (b->exec) {
    CEED_CUDA_CHECK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return CEED_OK;
  }
  return batch_launch_direct(b, (cudaStream_t)stream);
}

extern "C" int ceed_batch_status(ceed_batch_t b, void *stream) {
  if (!b) return fail(CEED_ERR_INVALID, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  CEED_CUDA_CHECK(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  if (err) {  // a bounded wait gave up: reset the barrier state for the next launch
    CEED_CUDA_CHECK(cudaMemsetAsync(b->d_sync, 0, 4 * sizeof(unsigned), s));
    CEED_CUDA_CHECK(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
    CEED_CUDA_CHECK(cudaStreamSynchronize(s));
    return fail(CEED_ERR_TIMEOUT, "a batched launch hit its grid-barrier or copy time limit");
  }
  return CEED_OK;
}

extern "C" int ceed_batch_info(ceed_batch_t b, int32_t *threads, int32_t *stage, uint32_t *grid) {
  if (!b) return fail(CEED_ERR_INVALID, "null batch");
  if (threads) *threads = b->L.threads;
  if (stage) *stage = b->L.stage;
  if (grid) *grid = b->grid;
  return CEED_OK;
}

extern "C" int ceed_batch_autotune(ceed_batch_t b, float *best_ms, void *stream) {
  if (!b) return fail(CEED_ERR_INVALID, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CEED_CUDA_CHECK(cudaEventCreate(&e0));
  CEED_CUDA_CHECK(cudaEventCreate(&e1));
  BatchLaunch best = b->L;
  float best_t = 1e30f;
  int maxq = 0;
  for (int k = 0; k < b->n; ++k) maxq = std::max(maxq, b->meshes[k]->Q);
  const int cand_threads[3] = {128, 192, 256};
  for (int ti = 0; ti < 3; ++ti) {
    if (cand_threads[ti] < maxq * maxq) continue;
    for (int stage = 0; stage <= 1; ++stage) {
      b->L = BatchLaunch{cand_threads[ti], stage, 0};
      if (batch_launch_direct(b, s) != CEED_OK) continue;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) batch_launch_direct(b, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= 3;
      if (ms < best_t) {
        best_t = ms;
        best = b->L;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->L = best;
  if (best_ms) *best_ms = best_t;
  if (int st = ceed_batch_status(b, stream)) return st;
  return build_graph(b);
}

extern "C" int ceed_batch_destroy(ceed_batch_t b) {
  if (!b) return CEED_OK;
  cudaDeviceSynchronize();
  drop_graph(b);
  cudaFree(b->d_sync);
  cudaFree(b->d_err);
  delete b;
  return CEED_OK;
}
