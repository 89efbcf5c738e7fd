// Fused Jacobi-PCG iteration: the whole iteration -- q = A p over every colour, alpha, the x and r
// updates with the r.z and r.r sums, beta and the p update -- in ONE persistent kernel, which runs
// a batch of iterations per launch (paper Section 1: CG on the matrix-free operator with a cheap
// preconditioner; Section 2.4: the Krylov updates are memory-bound streaming work; Section 3: fusing
// the operator's steps into one kernel removes global temporaries and launch gaps).
//
// The grid is launched cooperatively with as many blocks as can be resident at once, so that grid
// barriers (bounded waits, as in the batched kernel) can separate the colours of the atomic-free
// scatter and the phases of the iteration.  Every reduction has a fixed order: each block adds its
// share in a fixed sequence, and every block then sums the blocks' partials in block order itself,
// so all blocks hold the same alpha and beta and take the same stopping decision without another
// barrier.  Block 0 publishes the scalars for the host.  The update stores z = D^{-1} r for the p
// update (as many bytes as reading r and D^{-1} there, one FP64 product less per entry).
#pragma once

#include "batch.cuh"
#include "cg_fused_api.h"

namespace ceedgb {

struct CgFusedArgs {
  ApplyArgs a;                               // masked apply q = A p (x = p, y = q, ncol = 1)
  int64_t cstart[CGF_MAX_COLORS + 1];        // colour-sorted element ranges
  int ncolors;
  double *x, *r, *p, *q;
  double *z;                                 // z = D^{-1} r of the current iteration (written, read once)
  const double *dinv;
  int64_t n;
  double *part;                              // [3][gridDim]: p.q, r.z, r.r partials per block
  CgScalars *sc;
  unsigned *sync;                            // grid barrier state
  long long grid_wait;
  int iters;                                 // iterations this launch may run
  int fixed;                                 // 1: run them all (no tolerance stop)
};

// sum of v over the block's threads, in a fixed order (the result is valid in every thread)
__device__ __forceinline__ double cgf_block_sum(double v, double *red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();  // red is free (earlier readers are done)
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// sum of the G block partials part[0 .. G-1] in a fixed order, computed by every block
__device__ __forceinline__ double cgf_sum_partials(const double *part, int G, double *red) {
  double a = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) a += __ldcg(part + b);
  return cgf_block_sum(a, red);
}

template <int P, int Q, int OP, typename T, typename TQ>
__device__ __forceinline__ void cg_fused_body(const CgFusedArgs &g, const OpTab<T> &tab, unsigned char *smem_raw) {
  __shared__ double dsh;                    // this block's p.q partial of the current apply
  __shared__ double red[APPLY_MAX_THREADS / 32];
  __shared__ int ok_sh;
  __shared__ uint64_t nobar[1];
  const int G = gridDim.x;
  const int tid = threadIdx.x;
  CgScalars *sc = g.sc;
  // scalars at entry (written by the host or an earlier launch; block 0 updates sc only after the
  // first grid barrier, which every block reaches after these reads)
  if (sc->done) return;
  double rz = sc->rz;
  const double tol2 = sc->tol2, bb = sc->bb;
  int iters = sc->iters;
  const int64_t stride = (int64_t)G * blockDim.x;

  for (int it = 0; it < g.iters; ++it) {
    // ---- q = A p, colour by colour; each block adds p_i q_i over the nodes whose final value it writes
    if (tid == 0) dsh = 0.0;
    __syncthreads();
    ApplyArgs a = g.a;
    a.dot_sh = &dsh;
    for (int c = 0; c < g.ncolors; ++c) {
      a.e_begin = g.cstart[c];
      a.e_count = g.cstart[c + 1] - a.e_begin;
      const int64_t nwork = (a.e_count + a.ne - 1) / a.ne;
      for (int64_t v = blockIdx.x; v < nwork; v += G) {
        apply_block<P, Q, OP, T, TQ, false, true>(a, tab, v, smem_raw, nobar);
        __syncthreads();  // shared memory is reused by the next element block
      }
      if (c + 1 == g.ncolors && tid == 0) g.part[blockIdx.x] = dsh;
      if (!grid_barrier(g.sync, &sc->timeout, g.grid_wait, &ok_sh)) return;
    }
    // ---- alpha = r.z / p.q (every block sums the same partials in the same order)
    const double pq = cgf_sum_partials(g.part, G, red);
    const double alpha = rz / pq;
    if (!isfinite(alpha)) {
      if (blockIdx.x == 0 && tid == 0) {
        sc->pq = pq;
        sc->nonfinite = 1;
        sc->done = 1;
      }
      return;
    }
    // ---- x += alpha p; r -= alpha q; partial sums of r.z (z = D^{-1} r) and r.r.  Four strided
    // entries per trip keep enough loads in flight to stream at HBM rate; vectors written inside this
    // kernel are read through L2 (__ldcg).
    double arz[4] = {0.0, 0.0, 0.0, 0.0}, arr[4] = {0.0, 0.0, 0.0, 0.0};
    {
      int64_t k = (int64_t)blockIdx.x * blockDim.x + tid;
      for (; k + 3 * stride < g.n; k += 4 * stride) {
        double pk[4], xk[4], rk[4], qk[4], dk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t kk = k + u * stride;
          pk[u] = __ldcg(g.p + kk);
          xk[u] = __ldcg(g.x + kk);
          rk[u] = __ldcg(g.r + kk);
          qk[u] = __ldcg(g.q + kk);
          dk[u] = __ldg(g.dinv + kk);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t kk = k + u * stride;
          g.x[kk] = xk[u] + alpha * pk[u];
          const double rn = rk[u] - alpha * qk[u];
          g.r[kk] = rn;
          const double zn = dk[u] * rn;
          g.z[kk] = zn;
          arz[u] += rn * zn;
          arr[u] += rn * rn;
        }
      }
      for (; k < g.n; k += stride) {
        const double pk = __ldcg(g.p + k);
        g.x[k] = __ldcg(g.x + k) + alpha * pk;
        const double rn = __ldcg(g.r + k) - alpha * __ldcg(g.q + k);
        g.r[k] = rn;
        const double zn = __ldg(g.dinv + k) * rn;
        g.z[k] = zn;
        arz[0] += rn * zn;
        arr[0] += rn * rn;
      }
    }
    const double brz = cgf_block_sum((arz[0] + arz[1]) + (arz[2] + arz[3]), red);
    const double brr = cgf_block_sum((arr[0] + arr[1]) + (arr[2] + arr[3]), red);
    if (tid == 0) {
      g.part[G + blockIdx.x] = brz;
      g.part[2 * G + blockIdx.x] = brr;
    }
    if (!grid_barrier(g.sync, &sc->timeout, g.grid_wait, &ok_sh)) return;
    const double rz_new = cgf_sum_partials(g.part + G, G, red);
    const double rr = cgf_sum_partials(g.part + 2 * G, G, red);
    iters += 1;
    const bool nonfinite = !isfinite(rz_new) || !isfinite(rr);
    const bool stop = nonfinite || (!g.fixed && rr <= tol2 * bb);
    if (blockIdx.x == 0 && tid == 0) {
      sc->pq = pq;
      sc->alpha = alpha;
      sc->rz_new = rz_new;
      sc->rr = rr;
      sc->iters = iters;
      if (nonfinite) sc->nonfinite = 1;
      if (stop) sc->done = 1;
    }
    if (stop) return;  // stopped before the beta step (the reliable-update protocol relies on it)
    const double beta = rz_new / rz;
    rz = rz_new;
    if (blockIdx.x == 0 && tid == 0) {
      sc->beta = beta;
      sc->rz = rz;
    }
    // ---- p = z + beta p (z = D^{-1} r stored by the update: one FP64 FMA here instead of a product
    // and an FMA, at the same traffic -- z is written once and read once instead of reading r and
    // D^{-1}; GB300's FP64 pipe, not only HBM, bounds these streaming phases)
    {
      int64_t k = (int64_t)blockIdx.x * blockDim.x + tid;
      for (; k + 3 * stride < g.n; k += 4 * stride) {
        double zk[4], pk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          zk[u] = __ldcg(g.z + k + u * stride);
          pk[u] = __ldcg(g.p + k + u * stride);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) g.p[k + u * stride] = fma(beta, pk[u], zk[u]);
      }
      for (; k < g.n; k += stride) g.p[k] = fma(beta, __ldcg(g.p + k), __ldcg(g.z + k));
    }
    if (!grid_barrier(g.sync, &sc->timeout, g.grid_wait, &ok_sh)) return;
  }
}

// register caps of the fused iteration (measured at 64^3, p = 7 on the GB300 against the separate
// kernels, ms per iteration: FP32 operator 3.18 vs 3.47, FP64 14.81 vs 14.73 (uncapped: 15.9))
#ifndef CGF_F32_MAX_REGS
#define CGF_F32_MAX_REGS 96
#endif
#ifndef CGF_F64_MAX_REGS
#define CGF_F64_MAX_REGS 96
#endif
// Every instantiation runs under a register cap (blocks of at most 256 threads): the persistent body
// would otherwise hold more registers than the stand-alone apply kernel, i.e. fewer resident warps
// (FP32 operator: 124 uncapped, 16 warps per SM)
template <int P, int Q, int OP, typename T, typename TQ, int REGS>
__global__ void __maxnreg__(REGS) cg_fused_kernel(const CgFusedArgs g, const OpTab<T> tab) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cg_fused_body<P, Q, OP, T, TQ>(g, tab, smem_raw);
}

template <typename T>
constexpr int cgf_max_regs() {
  return std::is_same<T, DF>::value ? APPLY_DF_MAX_REGS
         : std::is_same<T, float>::value ? CGF_F32_MAX_REGS
                                         : CGF_F64_MAX_REGS;
}

// Launch `iters` fused iterations of one (P, op, T, TQ) instantiation (GLL collocated); `ne`
// elements per block of work.  The grid is every block that can be resident (cooperative launch).
template <int P, int OP, typename T, typename TQ>
int launch_cg_fused(const CgFusedArgs &gin, const OpTab<T> &tab, int ne, cudaStream_t s, unsigned *grid_out) {
  constexpr int Q = P;
  constexpr int REGS = cgf_max_regs<T>();
  if (ne < 1 || ne > max_elems_per_block<Q>() || ne > APPLY_MAX_NE) return fail(CEED_ERR_INVALID, "bad elements per block");
  const size_t smem = (size_t)ne * apply_elem_smem<P, Q, OP, T, TQ, false>();
  const void *kfn = (const void *)cg_fused_kernel<P, Q, OP, T, TQ, REGS>;
  if (int st = ensure_dynamic_smem(kfn, smem)) return st;
  const int threads = Q * Q * ne;
  int per_sm = 0, dev = 0, nsm = 0;
  CEED_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem));
  CEED_CUDA_CHECK(cudaGetDevice(&dev));
  CEED_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return fail(CEED_ERR_UNSUPPORTED, "fused CG kernel does not fit on an SM");
  const unsigned grid = (unsigned)std::min(per_sm * nsm, CGF_MAX_GRID);
  CgFusedArgs g = gin;
  g.a.ne = ne;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CEED_CUDA_CHECK(cudaLaunchKernelEx(&cfg, cg_fused_kernel<P, Q, OP, T, TQ, REGS>, g, tab));
  if (grid_out) *grid_out = grid;
  return CEED_OK;
}

// Dispatch on P (GLL collocated, so Q = P) for one (op, T, TQ).
template <int OP, typename T, typename TQ>
int dispatch_cg_fused(int P, const CgFusedArgs &g, const OpTab<T> &tab, int ne, cudaStream_t s, unsigned *grid) {
  switch (P) {
    case 2: return launch_cg_fused<2, OP, T, TQ>(g, tab, ne, s, grid);
    case 3: return launch_cg_fused<3, OP, T, TQ>(g, tab, ne, s, grid);
    case 4: return launch_cg_fused<4, OP, T, TQ>(g, tab, ne, s, grid);
    case 5: return launch_cg_fused<5, OP, T, TQ>(g, tab, ne, s, grid);
    case 6: return launch_cg_fused<6, OP, T, TQ>(g, tab, ne, s, grid);
    case 7: return launch_cg_fused<7, OP, T, TQ>(g, tab, ne, s, grid);
    case 8: return launch_cg_fused<8, OP, T, TQ>(g, tab, ne, s, grid);
    case 9: return launch_cg_fused<9, OP, T, TQ>(g, tab, ne, s, grid);
    default: return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
  }
}

}  // namespace ceedgb
