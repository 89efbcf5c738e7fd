// Batched apply: several independent meshes (different polynomial orders allowed) in ONE persistent
// launch.  Each thread block loops over the colours; within a colour it takes every G-th block of
// work across all meshes (G = blocks in the grid), and a grid-wide barrier separates colours so that
// the atomic-free scatter stays race-free.  The grid is sized to what is co-resident on the GPU;
// the barrier's wait is bounded (a timeout is recorded instead of hanging).
#pragma once

#include <algorithm>
#include <cstring>

#include "apply_kernel.cuh"

namespace ceedgb {

constexpr int BATCH_MAX = 4;
constexpr int BATCH_MAX_COLORS = 16;

struct BatchMesh {
  ApplyArgs a;                              // e_begin / e_count set per colour inside the kernel
  int P, Q, ncolors;
  int64_t cstart[BATCH_MAX_COLORS + 1];     // colour-sorted element ranges
};

template <typename T>
struct BatchArgs {
  int n, max_colors;
  unsigned *sync;                           // [0] arrivals, [1] generation
  int *err;
  long long grid_wait;                      // polls of the grid barrier before it gives up
  BatchMesh m[BATCH_MAX];
  OpTab<T> tab[BATCH_MAX];
};

// Bounded grid barrier (sense by generation counter).  Returns false on timeout.
__device__ __forceinline__ bool grid_barrier(unsigned *sync, int *err, long long limit, int *ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *vgen = sync + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(sync, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(sync, 0u);
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (++it > limit) {
          ok = 0;
          *err = CEED_ERR_TIMEOUT;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

template <int OP, typename T, typename TQ, bool STAGE, bool COLLOC>
__device__ __forceinline__ void batch_body(const BatchArgs<T> &b, unsigned char *smem_raw) {
  __shared__ uint64_t bar[STAGE ? APPLY_MAX_NE : 1];
  __shared__ int ok_sh;
  // the 1D tables of the mesh being processed, copied from the parameter block into shared memory
  // (indexing the parameter block by a run-time mesh slot would cost registers in every pass)
  __shared__ __align__(16) T tab_words[sizeof(OpTab<T>) / sizeof(T)];
  const OpTab<T> &tab = *reinterpret_cast<const OpTab<T> *>(tab_words);
  int cur_m = -1;
  for (int c = 0; c < b.max_colors; ++c) {
    int64_t nb[BATCH_MAX], total = 0;
#pragma unroll
    for (int m = 0; m < BATCH_MAX; ++m) {
      nb[m] = 0;
      if (m < b.n && c < b.m[m].ncolors) {
        const int64_t cnt = b.m[m].cstart[c + 1] - b.m[m].cstart[c];
        nb[m] = (cnt + b.m[m].a.ne - 1) / b.m[m].a.ne;
      }
      total += nb[m];
    }
    for (int64_t v = blockIdx.x; v < total; v += gridDim.x) {
      int m = 0;
      int64_t base = 0;
      while (v >= base + nb[m]) {
        base += nb[m];
        ++m;
      }
      ApplyArgs a = b.m[m].a;
      a.e_begin = b.m[m].cstart[c];
      a.e_count = b.m[m].cstart[c + 1] - a.e_begin;
      const int64_t blk = v - base;
      if (m != cur_m) {
        __syncthreads();
        const T *src = reinterpret_cast<const T *>(&b.tab[m]);
        for (int w = threadIdx.x; w < (int)(sizeof(OpTab<T>) / sizeof(T)); w += blockDim.x) tab_words[w] = src[w];
        __syncthreads();
        cur_m = m;
      }
#define CEEDGB_BCASE(PP)                                                                                         \
  case PP:                                                                                                      \
    apply_block<PP, COLLOC ? PP : PP + 1, OP, T, TQ, STAGE>(a, tab, blk, smem_raw, bar);                  \
    break;
      switch (b.m[m].P) {
        CEEDGB_BCASE(2)
        CEEDGB_BCASE(3)
        CEEDGB_BCASE(4)
        CEEDGB_BCASE(5)
        CEEDGB_BCASE(6)
        CEEDGB_BCASE(7)
        CEEDGB_BCASE(8)
        CEEDGB_BCASE(9)
        default:
          break;
      }
#undef CEEDGB_BCASE
      __syncthreads();  // shared memory is reused by the next block of work
    }
    if (c + 1 < b.max_colors && !grid_barrier(b.sync, b.err, b.grid_wait, &ok_sh)) return;
  }
}

template <int OP, typename T, typename TQ, bool STAGE, bool COLLOC>
__global__ void __launch_bounds__(APPLY_MAX_THREADS) batch_kernel(const BatchArgs<T> b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  batch_body<OP, T, TQ, STAGE, COLLOC>(b, smem_raw);
}

// Shared memory per thread block for a mesh with P nodes / Q points when blocks have `threads` threads.
template <int OP, typename T, typename TQ, bool STAGE>
size_t batch_smem_for(int P, int Q, int threads) {
  const int slots = (threads + Q * Q - 1) / (Q * Q);
  size_t eb = 0;
#define CEEDGB_S(PP)                                                                              \
  if (P == PP) eb = (Q == PP) ? apply_elem_smem<PP, PP, OP, T, TQ, STAGE>()                       \
                              : apply_elem_smem<PP, PP + 1, OP, T, TQ, STAGE>();
  CEEDGB_S(2) CEEDGB_S(3) CEEDGB_S(4) CEEDGB_S(5) CEEDGB_S(6) CEEDGB_S(7) CEEDGB_S(8) CEEDGB_S(9)
#undef CEEDGB_S
  return (size_t)slots * eb;
}


// Launch one batched apply (host side).  `launch` lists the meshes' apply requests.
template <int OP, typename T, typename TQ>
int launch_batch(int n, ceed_mesh_t const *meshes, const ApplyReq *reqs, const OpTab<T> *const *tabs,
                 unsigned *sync, int *err, const BatchLaunch &L, cudaStream_t s, unsigned *grid_used) {
  BatchArgs<T> b;
  std::memset(&b, 0, sizeof(b));
  b.n = n;
  b.sync = sync;
  b.err = err;
  b.grid_wait = grid_wait_limit();
  size_t smem = 0;
  const bool colloc = meshes[0]->Q == meshes[0]->P;
  for (int k = 0; k < n; ++k) {
    ceed_mesh_t m = meshes[k];
    if ((m->Q == m->P) != colloc) return fail(CEED_ERR_UNSUPPORTED, "a batch mixes quadrature rules");
    if (m->n_colors > BATCH_MAX_COLORS) return fail(CEED_ERR_UNSUPPORTED, "too many colours for a batch");
    BatchMesh &bm = b.m[k];
    bm.P = m->P;
    bm.Q = m->Q;
    bm.ncolors = m->n_colors;
    for (int c = 0; c <= m->n_colors; ++c) bm.cstart[c] = m->color_start[c];
    bm.a.emap = m->d_emap;
    bm.a.qdata = reqs[k].qdata;
    bm.a.x = reqs[k].x;
    bm.a.y = reqs[k].y;
    bm.a.ncol = reqs[k].ncol;
    bm.a.masked = reqs[k].masked;
    bm.a.ne = L.threads / (m->Q * m->Q);
    if (bm.a.ne < 1) return fail(CEED_ERR_INVALID, "block too small for this order");
    bm.a.err = err;
    bm.a.wait_limit = copy_wait_limit();
    bm.a.estride = qdata_estride(OP, sizeof(TQ), m->Q);
    bm.a.dot_part = nullptr;
    bm.a.dot_base = 0;
    bm.a.dot_sh = nullptr;
    b.tab[k] = *tabs[k];
    b.max_colors = std::max(b.max_colors, m->n_colors);
    const size_t sm = L.stage ? batch_smem_for<OP, T, TQ, true>(m->P, m->Q, L.threads)
                              : batch_smem_for<OP, T, TQ, false>(m->P, m->Q, L.threads);
    smem = std::max(smem, sm);
  }
  auto go = [&](auto kernel) -> int {
    CEED_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    CEED_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, L.threads, smem));
    CEED_CUDA_CHECK(cudaGetDevice(&dev));
    CEED_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(CEED_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    unsigned grid = (unsigned)(per_sm * nsm);
    if (L.grid > 0 && L.grid < grid) grid = L.grid;
    // cooperative launch: the runtime refuses it unless every block of the grid can be resident at
    // once, which is what the grid barrier between colours relies on (the barrier's bounded wait
    // stays as a second line of defence)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(L.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CEED_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kernel, b));
    if (grid_used) *grid_used = grid;
    return CEED_OK;
  };
  // (the double-float operator included: unlike its single-mesh kernel it runs fastest without a
  // register cap here -- 7.1 / 7.8 GDOF/s at 1 / 4 right-hand sides against 6.1 at 128 registers)
  if (colloc) return L.stage ? go(batch_kernel<OP, T, TQ, true, true>) : go(batch_kernel<OP, T, TQ, false, true>);
  return L.stage ? go(batch_kernel<OP, T, TQ, true, false>) : go(batch_kernel<OP, T, TQ, false, false>);
}

}  // namespace ceedgb
