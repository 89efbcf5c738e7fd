// Jacobi-preconditioned conjugate gradients on the matrix-free operator (paper Section 1: CG
// with a cheap preconditioner; Section 2.4: Krylov updates are memory-bound streaming kernels),
// plus FP64-outer / low-precision-inner iterative refinement.
//
// All scalars live on the device; every kernel after convergence is a no-op (it reads the done
// flag), so a batch of iterations can be queued without host round trips.  Reductions are
// deterministic: a fixed grid writes per-block partial sums that one block adds in fixed order.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "cg_fused.cuh"
#include "internal.h"

namespace ceedgb {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

static int red_blocks(int64_t n) {
  int64_t b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return (int)b;
}

using Scalars = CgScalars;

__device__ __forceinline__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Grid-stride loops below take four strided entries per trip (independent loads in flight,
// independent partial sums); the summation order is fixed by (n, grid) so results are reproducible.
#define CEEDGB_GRID4(BODY)                                                                     \
  {                                                                                            \
    const int64_t stride_ = (int64_t)gridDim.x * blockDim.x;                                   \
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;                                \
    for (; i + 3 * stride_ < n; i += 4 * stride_) {                                            \
      { const int u_ = 0; (void)u_; const int64_t k = i; BODY }                                \
      { const int u_ = 1; (void)u_; const int64_t k = i + stride_; BODY }                      \
      { const int u_ = 2; (void)u_; const int64_t k = i + 2 * stride_; BODY }                  \
      { const int u_ = 3; (void)u_; const int64_t k = i + 3 * stride_; BODY }                  \
    }                                                                                          \
    for (; i < n; i += stride_) { const int u_ = 0; (void)u_; const int64_t k = i; BODY }      \
  }

__global__ void dot_partial_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                   double *__restrict__ part, const Scalars *sc) {
  __shared__ double sh[RED_THREADS];
  if (sc && sc->done) return;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  CEEDGB_GRID4(a[u_] += x[k] * y[k];)
  double t = block_sum((a[0] + a[1]) + (a[2] + a[3]), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Sums nb partials in fixed order into *out.
__global__ void sum_partials_kernel(const double *__restrict__ part, int nb, double *out) {
  __shared__ double sh[RED_THREADS];
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += RED_THREADS) a += part[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) *out = a;
}

// Launched with 1024 threads: sums nb partials (up to one per element) in a fixed order.
__global__ void finalize_alpha_kernel(const double *__restrict__ part, int64_t nb, Scalars *sc) {
  __shared__ double sh[1024];
  if (sc->done) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int64_t i = threadIdx.x;
  for (; i + 3 * 1024 < nb; i += 4 * 1024) {
    a0 += part[i];
    a1 += part[i + 1024];
    a2 += part[i + 2048];
    a3 += part[i + 3072];
  }
  for (; i < nb; i += 1024) a0 += part[i];
  sh[threadIdx.x] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  for (int st = 512; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  const double a = sh[0];
  if (threadIdx.x == 0) {
    sc->pq = a;
    sc->alpha = sc->rz / a;
    if (!finite(sc->alpha)) {
      sc->nonfinite = 1;
      sc->done = 1;
    }
  }
}

// x += alpha p; r -= alpha q; z = dinv r; partials of r.z and r.r
__global__ void update_kernel(double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                              const double *__restrict__ p, const double *__restrict__ q,
                              const double *__restrict__ dinv, int64_t n, double *__restrict__ part_rz,
                              double *__restrict__ part_rr, const Scalars *sc) {
  __shared__ double sh[RED_THREADS];
  if (sc->done) return;
  const double alpha = sc->alpha;
  double arz[4] = {0.0, 0.0, 0.0, 0.0}, arr[4] = {0.0, 0.0, 0.0, 0.0};
  CEEDGB_GRID4({
    x[k] += alpha * p[k];
    const double ri = r[k] - alpha * q[k];
    r[k] = ri;
    const double zi = dinv[k] * ri;
    z[k] = zi;
    arz[u_] += ri * zi;
    arr[u_] += ri * ri;
  })
  const double trz = block_sum((arz[0] + arz[1]) + (arz[2] + arz[3]), sh);
  const double trr = block_sum((arr[0] + arr[1]) + (arr[2] + arr[3]), sh);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = trz;
    part_rr[blockIdx.x] = trr;
  }
}

__global__ void finalize_beta_kernel(const double *__restrict__ part_rz, const double *__restrict__ part_rr, int nb,
                                     Scalars *sc, int fixed) {
  __shared__ double sh[RED_THREADS];
  if (sc->done) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += RED_THREADS) {
    a += part_rz[i];
    b += part_rr[i];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    sc->rz_new = a;
    sc->rr = b;
    sc->iters += 1;
    if (!finite(a) || !finite(b)) {
      sc->nonfinite = 1;
      sc->done = 1;
      return;
    }
    if (!fixed && b <= sc->tol2 * sc->bb) {
      sc->done = 1;
      return;
    }
    sc->beta = a / sc->rz;
    sc->rz = a;
  }
}

// Residual replacement of the reliable-update CG, after an iteration that stopped before its beta
// step: rz and rr of the replaced residual from partials, beta = rz_new / rz_old (the p update
// that follows uses the true residual's z).
__global__ void replace_finalize_kernel(const double *__restrict__ part_rz, const double *__restrict__ part_rr,
                                        int nb, Scalars *sc) {
  __shared__ double sh[RED_THREADS];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += RED_THREADS) {
    a += part_rz[i];
    b += part_rr[i];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    sc->beta = a / sc->rz;
    sc->rz = a;
    sc->rr = b;
    sc->nonfinite = (!finite(a) || !finite(b) || !finite(sc->beta)) ? 1 : 0;
    sc->done = sc->nonfinite || b == 0.0;
  }
}

__global__ void pupdate_kernel(double *__restrict__ p, const double *__restrict__ z, int64_t n, const Scalars *sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  CEEDGB_GRID4(p[k] = z[k] + beta * p[k];)
}

// CG start from r (already holding the initial residual): z = dinv r, p = z (set_p), partials of
// r.z, r.r.  Without set_p (residual replacement of the reliable-update CG) the direction p is kept.
__global__ void start_kernel(const double *__restrict__ r, double *__restrict__ z, double *__restrict__ p,
                             const double *__restrict__ dinv, int64_t n, double *__restrict__ part_rz,
                             double *__restrict__ part_rr, int set_p) {
  __shared__ double sh[RED_THREADS];
  double arz[4] = {0.0, 0.0, 0.0, 0.0}, arr[4] = {0.0, 0.0, 0.0, 0.0};
  CEEDGB_GRID4({
    const double ri = r[k];
    const double zi = dinv[k] * ri;
    z[k] = zi;
    if (set_p) p[k] = zi;
    arz[u_] += ri * zi;
    arr[u_] += ri * ri;
  })
  const double trz = block_sum((arz[0] + arz[1]) + (arz[2] + arz[3]), sh);
  const double trr = block_sum((arr[0] + arr[1]) + (arr[2] + arr[3]), sh);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = trz;
    part_rr[blockIdx.x] = trr;
  }
}

// rz, rr from partials; bb = rr * scale (scale = 1: relative to the initial residual) or kept;
// tol2 set by the host.  done if the start already meets the tolerance.
__global__ void start_finalize_kernel(const double *__restrict__ part_rz, const double *__restrict__ part_rr, int nb,
                                      Scalars *sc, int set_bb_from_rr, int fixed) {
  __shared__ double sh[RED_THREADS];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += RED_THREADS) {
    a += part_rz[i];
    b += part_rr[i];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    sc->rz = a;
    sc->rr = b;
    if (set_bb_from_rr) sc->bb = b;
    sc->iters = 0;
    sc->timeout = 0;
    sc->nonfinite = (!finite(a) || !finite(b)) ? 1 : 0;
    sc->done = sc->nonfinite || (!fixed && b <= sc->tol2 * sc->bb) || b == 0.0;
  }
}

// out = b - Ax (elementwise), partials of out.out
__global__ void residual_kernel(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ out,
                                int64_t n, double *__restrict__ part) {
  __shared__ double sh[RED_THREADS];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  CEEDGB_GRID4({
    const double v = b[k] - Ax[k];
    out[k] = v;
    a[u_] += v * v;
  })
  const double t = block_sum((a[0] + a[1]) + (a[2] + a[3]), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void axpy_kernel(double *__restrict__ x, const double *__restrict__ d, int64_t n) {
  CEEDGB_GRID4(x[k] += d[k];)
}

__global__ void invert_kernel(double *__restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = 1.0 / d[i];
}

__global__ void zero_kernel(double *__restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = 0.0;
}

__global__ void copy_kernel(double *__restrict__ d, const double *__restrict__ s, int64_t n) {
  CEEDGB_GRID4(d[k] = s[k];)
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Work {
  double *r_out, *d, *r, *z, *p, *q, *dinv, *part1, *part2;
  double *r_old;    // flexible CG: residual of the previous iteration
  double *pq_part;  // per-block partial sums of p . q written by the fused apply
  double *fpart;    // fused iteration: per-block partials [3][CGF_MAX_GRID]
  unsigned *fsync;  // fused iteration: grid barrier state
  Scalars *sc;
};

static size_t layout(int64_t n, int64_t n_elem, bool mixed, char *base, Work *w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *ptr = base ? base + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  const size_t vb = (size_t)n * sizeof(double);
  Work t{};
  t.r = (double *)take(vb);
  t.z = (double *)take(vb);
  t.p = (double *)take(vb);
  t.q = (double *)take(vb);
  t.dinv = (double *)take(vb);
  (void)mixed;
  t.r_out = (double *)take(vb);
  t.d = (double *)take(vb);
  t.r_old = (double *)take(vb);
  t.pq_part = (double *)take((size_t)n_elem * sizeof(double));
  t.part1 = (double *)take(RED_MAX_BLOCKS * sizeof(double));
  t.part2 = (double *)take(RED_MAX_BLOCKS * sizeof(double));
  t.fpart = (double *)take(3 * CGF_MAX_GRID * sizeof(double));
  t.fsync = (unsigned *)take(4 * sizeof(unsigned));
  t.sc = (Scalars *)take(sizeof(Scalars));
  if (w) *w = t;
  return off;
}

static unsigned stream_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

static int read_scalars(Scalars *h, const Scalars *d, cudaStream_t s) {
  CEED_CUDA_CHECK(cudaMemcpyAsync(h, d, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  return CEED_OK;
}

// One PCG iteration on the device scalars (no host round trip): q = A p, alpha, x/r/z update, beta,
// p update.  no_stop: the tolerance test never ends the iteration (the host decides).
static int pcg_iteration(ceed_mesh_t m, const ApplyReq &op, double *y, const Work &w, int64_t n, bool no_stop,
                         cudaStream_t s) {
  const int nb = red_blocks(n);
  // q = A p.  FP64 operator: p . q is summed by the apply itself (each node's last writer adds
  // p_i q_i), saving two vector passes at no cost to the FP64-pipe-bound kernel.  FP32 operators
  // keep the separate reduction: with the fused sum (FP64 products and a block reduction inside
  // the FP32 kernel) the mixed CG at 64^3, p = 7 measured 3-9% slower than with the two passes.
  ApplyReq a = op;
  a.x = w.p;
  a.y = w.q;
  const bool fuse = (op.prec == CEED_F64);
  a.dot_part = fuse ? w.pq_part : nullptr;
  int64_t npart = 0;
  a.dot_n = &npart;
  if (int st = launch_apply(m, a, s)) return st;
  if (fuse) {
    finalize_alpha_kernel<<<1, 1024, 0, s>>>(w.pq_part, npart, w.sc);
  } else {
    dot_partial_kernel<<<nb, RED_THREADS, 0, s>>>(w.p, w.q, n, w.part1, w.sc);
    finalize_alpha_kernel<<<1, 1024, 0, s>>>(w.part1, nb, w.sc);
  }
  update_kernel<<<nb, RED_THREADS, 0, s>>>(y, w.r, w.z, w.p, w.q, w.dinv, n, w.part1, w.part2, w.sc);
  finalize_beta_kernel<<<1, RED_THREADS, 0, s>>>(w.part1, w.part2, nb, w.sc, no_stop ? 1 : 0);
  pupdate_kernel<<<stream_blocks(n), 256, 0, s>>>(w.p, w.z, n, w.sc);
  return CEED_OK;
}

// The fused iteration (cg_fused.cuh) covers the CG configuration of the paper's bake-off solves:
// diffusion, GLL-collocated quadrature, one component, FP64 / FP32 / BF16 / on-the-fly-geometry /
// double-float operators.  Other operators run the iteration as separate kernels (pcg_iteration).
static bool fused_supported(ceed_mesh_t m, const ApplyReq &op) {
  return op.op == CEED_OP_DIFFUSION && m->P == m->Q && op.ncol == 1 && m->n_colors <= CGF_MAX_COLORS &&
         (op.prec == CEED_F64 || op.prec == CEED_F32 || op.prec == CEED_BF16 || op.prec == CEED_F32_GEO ||
          op.prec == CEED_F64_DF);
}

// Up to `iters` PCG iterations in one fused launch (same device scalars and stopping rules as
// pcg_iteration; fixed: no tolerance stop).
static int fused_batch(ceed_mesh_t m, const ApplyReq &op, double *y, const Work &w, int64_t n, int iters, bool fixed,
                       cudaStream_t s) {
  CgFusedArgs g;
  std::memset(&g, 0, sizeof(g));
  const int qop = (op.prec == CEED_F32_GEO) ? OP_DIFF_GEO : CEED_OP_DIFFUSION;
  g.a.emap = m->d_emap;
  g.a.qdata = op.qdata;
  g.a.x = w.p;
  g.a.y = w.q;
  g.a.ncol = 1;
  g.a.masked = op.masked;
  g.a.err = m->d_err + 1;
  g.a.wait_limit = copy_wait_limit();
  g.a.estride = qdata_estride(qop, prec_size(op.prec), m->Q);
  for (int c = 0; c <= m->n_colors; ++c) g.cstart[c] = m->color_start[c];
  g.ncolors = m->n_colors;
  g.x = y;
  g.r = w.r;
  g.p = w.p;
  g.q = w.q;
  g.z = w.z;
  g.dinv = w.dinv;
  g.n = n;
  g.part = w.fpart;
  g.sc = w.sc;
  g.sync = w.fsync;
  g.grid_wait = grid_wait_limit();
  g.iters = iters;
  g.fixed = fixed ? 1 : 0;
  if (((uintptr_t)op.qdata & 15) != 0) return fail(CEED_ERR_INVALID, "qdata must be 16-byte aligned");
  CEED_CUDA_CHECK(cudaMemsetAsync(w.fsync, 0, 4 * sizeof(unsigned), s));  // barrier state (a timeout leaves it dirty)
  // elements per block: the apply variant chosen for this operator (autotuner or
  // ceed_set_apply_variant), else blocks of about 128 threads
  const ApplyChoice &tc = m->tuned[CEED_OP_DIFFUSION][op.prec];
  // a tuned brick variant says nothing about element blocks; the fused iteration keeps the element
  // kernel (at 64^3, p = 7 with the FP32 operator the persistent grid fits three brick blocks per SM
  // and measured 3.33 ms per iteration against 3.13)
  const int tuned = tc.stage < 2 ? tc.ne : 0;
  const int ne = tuned > 0 ? tuned : std::max(1, std::min(APPLY_MAX_NE, 128 / (m->Q * m->Q)));
  unsigned grid = 0;
  switch (op.prec) {
    case CEED_F64: return launch_cg_fused_f64(m, g, ne, s, &grid);
    case CEED_F64_DF: return launch_cg_fused_df(m, g, ne, s, &grid);
    default: return launch_cg_fused_f32(m, op.prec, g, ne, s, &grid);
  }
}

// Run PCG on A y = rhs (y starts at 0; rhs in w.r on entry), with the given operator.
// Stops when ||r|| <= tol ||ref|| (ref = rhs), or after max_iter iterations, or exactly `fixed` iterations.
// fused: whole iterations in the persistent kernel where the operator supports it.
static int pcg_run(ceed_mesh_t m, const ApplyReq &op, double *y, const Work &w, int64_t n, double tol, int max_iter,
                   int check_every, int fixed, cudaStream_t s, int *iters_out, int *nonfinite, bool fused = true,
                   int *fused_out = nullptr) {
  fused = fused && fused_supported(m, op);
  if (fused_out) *fused_out = fused ? 1 : 0;
  const int nb = red_blocks(n);
  Scalars h{};
  // tol2 and bb: bb comes from ||rhs||^2 (start_finalize with set_bb_from_rr)
  h.tol2 = tol * tol;
  CEED_CUDA_CHECK(cudaMemcpyAsync(&w.sc->tol2, &h.tol2, sizeof(double), cudaMemcpyHostToDevice, s));
  zero_kernel<<<stream_blocks(n), 256, 0, s>>>(y, n);
  start_kernel<<<nb, RED_THREADS, 0, s>>>(w.r, w.z, w.p, w.dinv, n, w.part1, w.part2, 1);
  start_finalize_kernel<<<1, RED_THREADS, 0, s>>>(w.part1, w.part2, nb, w.sc, 1, fixed > 0);
  CEED_CUDA_CHECK(cudaGetLastError());
  const int cap = fixed > 0 ? fixed : max_iter;
  int it = 0;
  while (it < cap) {
    const int batch = std::min(cap - it, fixed > 0 ? cap : check_every);
    if (fused) {
      if (int st = fused_batch(m, op, y, w, n, batch, fixed > 0, s)) return st;
    } else {
      for (int b = 0; b < batch; ++b)
        if (int st = pcg_iteration(m, op, y, w, n, fixed > 0, s)) return st;
    }
    CEED_CUDA_CHECK(cudaGetLastError());
    it += batch;
    if (int st = read_scalars(&h, w.sc, s)) return st;
    if (h.timeout) return fail(CEED_ERR_TIMEOUT, "a grid barrier of the fused CG iteration gave up");
    if (h.done) break;
  }
  if (fixed <= 0 || !h.done) {
    if (int st = read_scalars(&h, w.sc, s)) return st;
  }
  *iters_out = h.iters;
  *nonfinite = h.nonfinite;
  return CEED_OK;
}

// r_out = b - A x with the operator; returns ||r_out||^2 on the host.
static int residual(ceed_mesh_t m, const ApplyReq &op, const double *b, const double *x, double *Ax, double *r_out,
                    int64_t n, double *part, double *dsum, cudaStream_t s, double *rr) {
  ApplyReq a = op;
  a.x = x;
  a.y = Ax;
  if (int st = launch_apply(m, a, s)) return st;
  const int nb = red_blocks(n);
  residual_kernel<<<nb, RED_THREADS, 0, s>>>(b, Ax, r_out, n, part);
  sum_partials_kernel<<<1, RED_THREADS, 0, s>>>(part, nb, dsum);
  CEED_CUDA_CHECK(cudaGetLastError());
  CEED_CUDA_CHECK(cudaMemcpyAsync(rr, dsum, sizeof(double), cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  return CEED_OK;
}


// Jacobi-PCG on A x = b run with the low-precision operator `lo`, with reliable updates (residual
// replacement; Sleijpen and van der Vorst, Computing 56, 1996): x and every vector stay FP64.  The
// device stops an iteration before its beta step once the recurrence residual has fallen by `delta`
// since the last replacement (or has met the tolerance); the host then evaluates the true residual
// b - A x with the FP64 operator `hi`, stops if it meets tol, and otherwise puts it in place of the
// recurrence residual and completes the stopped step with it (z = D^{-1} r, beta = r.z / r.z_old,
// p = z + beta p), so the Krylov process is not restarted.  x holds the initial guess.  Counts:
// iterations, true-residual evaluations.
static int reliable_run(ceed_mesh_t m, const ApplyReq &hi, const ApplyReq &lo, const double *b, double *x,
                        const Work &w, int64_t n, double bb, double tol, double delta, int max_iter, int check_every,
                        cudaStream_t s, int *iters_out, int *evals_out, double *rel_out, int *nonfinite,
                        bool fused = true, int *fused_out = nullptr) {
  fused = fused && fused_supported(m, lo);
  if (fused_out) *fused_out = fused ? 1 : 0;
  const int nb = red_blocks(n);
  *iters_out = 0;
  *evals_out = 1;
  *nonfinite = 0;
  double rr = 0.0;
  if (int st = residual(m, hi, b, x, w.q, w.r, n, w.part1, &w.sc->rr_out, s, &rr)) return st;
  *rel_out = std::sqrt(rr / bb);
  if (!std::isfinite(rr)) {
    *nonfinite = 1;
    return CEED_OK;
  }
  if (*rel_out <= tol) return CEED_OK;
  // device stop threshold: rr <= tol2 * bb with tol2 = max(tol^2, delta^2 rr_ref / bb)
  auto set_stop = [&](double rr_ref) -> int {
    static_assert(offsetof(Scalars, tol2) == offsetof(Scalars, bb) + sizeof(double), "Scalars layout");
    const double v[2] = {bb, std::max(tol * tol, delta * delta * rr_ref / bb)};  // Scalars::bb, ::tol2
    CEED_CUDA_CHECK(cudaMemcpyAsync(&w.sc->bb, v, sizeof(v), cudaMemcpyHostToDevice, s));
    CEED_CUDA_CHECK(cudaStreamSynchronize(s));  // v lives on this stack frame
    return CEED_OK;
  };
  if (int st = set_stop(rr)) return st;
  start_kernel<<<nb, RED_THREADS, 0, s>>>(w.r, w.z, w.p, w.dinv, n, w.part1, w.part2, 1);
  start_finalize_kernel<<<1, RED_THREADS, 0, s>>>(w.part1, w.part2, nb, w.sc, 0, 0);
  CEED_CUDA_CHECK(cudaGetLastError());
  Scalars h{};
  int it = 0;
  // every batch completes at least one iteration (a replacement leaves done = 0), so the batch count
  // bound only guards against a stuck state
  for (int batches = 0; it < max_iter && batches <= max_iter; ++batches) {
    const int batch = std::min(max_iter - it, check_every);
    if (fused) {
      if (int st = fused_batch(m, lo, x, w, n, batch, false, s)) return st;
    } else {
      for (int k = 0; k < batch; ++k)
        if (int st = pcg_iteration(m, lo, x, w, n, false, s)) return st;
    }
    CEED_CUDA_CHECK(cudaGetLastError());
    if (int st = read_scalars(&h, w.sc, s)) return st;
    if (h.timeout) return fail(CEED_ERR_TIMEOUT, "a grid barrier of the fused CG iteration gave up");
    it = h.iters;  // completed iterations since the start (replacements do not reset the count)
    if (h.nonfinite) {
      *nonfinite = 1;
      break;
    }
    // the true residual is evaluated at every stop and at the cap, so *rel_out describes the final x
    if (!h.done && it < max_iter) continue;
    if (int st = residual(m, hi, b, x, w.q, w.r_out, n, w.part1, &w.sc->rr_out, s, &rr)) return st;
    *evals_out += 1;
    *rel_out = std::sqrt(rr / bb);
    if (!std::isfinite(rr)) {
      *nonfinite = 1;
      break;
    }
    if (*rel_out <= tol || !h.done) break;  // converged, or at the cap
    copy_kernel<<<stream_blocks(n), 256, 0, s>>>(w.r, w.r_out, n);
    if (int st = set_stop(rr)) return st;
    start_kernel<<<nb, RED_THREADS, 0, s>>>(w.r, w.z, w.p, w.dinv, n, w.part1, w.part2, 0);
    replace_finalize_kernel<<<1, RED_THREADS, 0, s>>>(w.part1, w.part2, nb, w.sc);
    pupdate_kernel<<<stream_blocks(n), 256, 0, s>>>(w.p, w.z, n, w.sc);
    CEED_CUDA_CHECK(cudaGetLastError());
  }
  *iters_out = it;
  return CEED_OK;
}

// ---------------------------------------------------------------- p-multigrid (V-cycle)
__global__ void cheb_init_kernel(double *__restrict__ x, double *__restrict__ r, double *__restrict__ d,
                                 const double *__restrict__ b, const double *__restrict__ q,
                                 const double *__restrict__ dinv, int64_t n, double inv_theta, int zero_x) {
  CEEDGB_GRID4({
    const double ri = zero_x ? b[k] : b[k] - q[k];
    if (zero_x) x[k] = 0.0;
    r[k] = ri;
    d[k] = inv_theta * dinv[k] * ri;
  })
}

// Chebyshev step (Saad, Iterative Methods, Chebyshev acceleration): x += d; r -= A d; d = c1 d + c2 D^{-1} r
__global__ void cheb_step_kernel(double *__restrict__ x, double *__restrict__ r, double *__restrict__ d,
                                 const double *__restrict__ q, const double *__restrict__ dinv, int64_t n, double c1,
                                 double c2) {
  CEEDGB_GRID4({
    const double di = d[k];
    x[k] += di;
    const double ri = r[k] - q[k];
    r[k] = ri;
    d[k] = c1 * di + c2 * dinv[k] * ri;
  })
}

__global__ void scale_kernel(double *__restrict__ v, const double *__restrict__ dinv, const double *__restrict__ w,
                             int64_t n, double f) {
  CEEDGB_GRID4(v[k] = f * dinv[k] * w[k];)
}

__global__ void scal_kernel(double *__restrict__ v, int64_t n, double f) { CEEDGB_GRID4(v[k] *= f;) }

__global__ void seed_kernel(double *__restrict__ v, int64_t n) {
  CEEDGB_GRID4({
    uint64_t z = (uint64_t)k * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[k] = 0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0);
  })
}

// FCG update: x += alpha p; r_old = r; r -= alpha q; partials of r.r
__global__ void fcg_update_kernel(double *__restrict__ x, double *__restrict__ r, double *__restrict__ r_old,
                                  const double *__restrict__ p, const double *__restrict__ q, int64_t n, double alpha,
                                  double *__restrict__ part) {
  __shared__ double sh[RED_THREADS];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  CEEDGB_GRID4({
    x[k] += alpha * p[k];
    const double ro = r[k];
    r_old[k] = ro;
    const double ri = ro - alpha * q[k];
    r[k] = ri;
    a[u_] += ri * ri;
  })
  const double t = block_sum((a[0] + a[1]) + (a[2] + a[3]), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void xpby_kernel(double *__restrict__ p, const double *__restrict__ z, int64_t n, double beta) {
  CEEDGB_GRID4(p[k] = z[k] + beta * p[k];)
}

struct PmgLevel {
  ceed_mesh_t mesh = nullptr;
  int64_t n = 0;
  ApplyReq op;              // smoothing operator (masked)
  double *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *q = nullptr, *dinv = nullptr;
  double *z = nullptr;      // Schwarz smoother: M r
  ceed_schwarz_t sw = nullptr;
  double lam = 1.0;
};

}  // namespace ceedgb

struct ceed_pmg_s {
  int L = 0;
  ceedgb::PmgLevel lv[4];
  ceed_pmg_opts o{};
  char *cwork = nullptr;     // coarse-level CG workspace
  ceedgb::Work cw;
  double *dsum = nullptr;    // device scalar
  double *part = nullptr;    // RED_MAX_BLOCKS partial sums
  std::vector<void *> allocs;
};

namespace ceedgb {

static double host_dot(const double *x, const double *y, int64_t n, double *part, double *dsum, cudaStream_t s,
                       int *st) {
  const int nb = red_blocks(n);
  dot_partial_kernel<<<nb, RED_THREADS, 0, s>>>(x, y, n, part, nullptr);
  sum_partials_kernel<<<1, RED_THREADS, 0, s>>>(part, nb, dsum);
  double h = 0.0;
  cudaError_t e = cudaMemcpyAsync(&h, dsum, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) *st = cuda_fail(e, "dot");
  return h;
}

__global__ void cheb_res_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ b,
                                const double *__restrict__ q, int64_t n, int zero_x) {
  CEEDGB_GRID4({
    r[k] = zero_x ? b[k] : b[k] - q[k];
    if (zero_x) x[k] = 0.0;
  })
}

// Chebyshev step with a preconditioner application z = M r: x += d; r -= A d (q = A d); then, after
// z = M r, d = c1 d + c2 z.
__global__ void cheb_xr_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ d,
                               const double *__restrict__ q, int64_t n) {
  CEEDGB_GRID4({
    x[k] += d[k];
    r[k] -= q[k];
  })
}

__global__ void cheb_dir_kernel(double *__restrict__ d, const double *__restrict__ z, int64_t n, double c1, double c2) {
  CEEDGB_GRID4(d[k] = c1 * d[k] + c2 * z[k];)
}

// Chebyshev smoothing on M A with the Schwarz smoother M (same recurrence as the Jacobi version).
static int pmg_cheb_schwarz(ceed_pmg_s *P, int l, int degree, double lo, double hi, bool zero_x, cudaStream_t s) {
  PmgLevel &L = P->lv[l];
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (!zero_x) {
    ApplyReq a = L.op;
    a.x = L.x;
    a.y = L.q;
    if (int st = launch_apply(L.mesh, a, s)) return st;
  }
  cheb_res_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.x, L.r, L.b, L.q, L.n, zero_x);
  if (int st = launch_schwarz(L.sw, L.r, L.z, 1, s)) return st;
  cheb_dir_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.d, L.z, L.n, 0.0, 1.0 / theta);
  for (int k = 0; k < degree; ++k) {
    if (k == degree - 1) {
      axpy_kernel<<<stream_blocks(L.n), 256, 0, s>>>(L.x, L.d, L.n);
      break;
    }
    ApplyReq a = L.op;
    a.x = L.d;
    a.y = L.q;
    if (int st = launch_apply(L.mesh, a, s)) return st;
    cheb_xr_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.x, L.r, L.d, L.q, L.n);
    if (int st = launch_schwarz(L.sw, L.r, L.z, 1, s)) return st;
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    cheb_dir_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.d, L.z, L.n, rho_new * rho, 2.0 * rho_new / delta);
    rho = rho_new;
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

// Chebyshev smoothing of A x = b on level l (x0 = 0 or the current x), `degree` products with A.
static int pmg_cheb(ceed_pmg_s *P, int l, int degree, double lo, double hi, bool zero_x, cudaStream_t s) {
  PmgLevel &L = P->lv[l];
  if (L.sw) return pmg_cheb_schwarz(P, l, degree, lo, hi, zero_x, s);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (!zero_x) {
    ApplyReq a = L.op;
    a.x = L.x;
    a.y = L.q;
    if (int st = launch_apply(L.mesh, a, s)) return st;
  }
  cheb_init_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.x, L.r, L.d, L.b, L.q, L.dinv, L.n, 1.0 / theta, zero_x);
  for (int k = 0; k < degree; ++k) {
    if (k == degree - 1) {
      axpy_kernel<<<stream_blocks(L.n), 256, 0, s>>>(L.x, L.d, L.n);
      break;
    }
    ApplyReq a = L.op;
    a.x = L.d;
    a.y = L.q;
    if (int st = launch_apply(L.mesh, a, s)) return st;
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    cheb_step_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.x, L.r, L.d, L.q, L.dinv, L.n, rho_new * rho,
                                                              2.0 * rho_new / delta);
    rho = rho_new;
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

// V-cycle on level l: lv[l].x approximates A_l^{-1} lv[l].b.
static int pmg_vcycle(ceed_pmg_s *P, int l, cudaStream_t s) {
  PmgLevel &L = P->lv[l];
  if (l == P->L - 1) {  // coarsest: Jacobi-PCG to coarse_tol
    copy_kernel<<<stream_blocks(L.n), 256, 0, s>>>(P->cw.r, L.b, L.n);
    int iters = 0, nonfin = 0;
    if (int st = pcg_run(L.mesh, L.op, L.x, P->cw, L.n, P->o.coarse_tol, P->o.coarse_max_iter, 50, 0, s, &iters,
                         &nonfin))
      return st;
    return CEED_OK;
  }
  const double hi = 1.1 * L.lam, lo = hi / P->o.smooth_ratio;
  if (int st = pmg_cheb(P, l, P->o.smooth_degree, lo, hi, true, s)) return st;
  {  // residual r = b - A x
    ApplyReq a = L.op;
    a.x = L.x;
    a.y = L.q;
    if (int st = launch_apply(L.mesh, a, s)) return st;
    residual_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.b, L.q, L.r, L.n, P->part);
  }
  PmgLevel &C = P->lv[l + 1];
  if (int st = launch_restrict(C.mesh, L.mesh, L.r, C.b, s)) return st;
  if (int st = pmg_vcycle(P, l + 1, s)) return st;
  if (int st = launch_prolong(C.mesh, L.mesh, C.x, L.x, 1, s)) return st;
  return pmg_cheb(P, l, P->o.smooth_degree, lo, hi, false, s);
}

// Flexible CG (Notay): beta = (z_{k+1} . (r_{k+1} - r_k)) / (z_k . r_k), preconditioned by one V-cycle.
static int fcg_run(ceed_mesh_t m, const ApplyReq &op64, ceed_pmg_s *P, double *x, const double *b, const Work &w,
                   int64_t n, double tol, int max_iter, cudaStream_t s, int *iters_out, int *nonfin) {
  int st = CEED_OK;
  const double bb = host_dot(b, b, n, w.part1, &w.sc->bb_out, s, &st);
  if (st) return st;
  zero_kernel<<<stream_blocks(n), 256, 0, s>>>(x, n);
  copy_kernel<<<stream_blocks(n), 256, 0, s>>>(w.r, b, n);
  PmgLevel &F = P->lv[0];
  auto precond = [&](const double *r, double *z) -> int {
    copy_kernel<<<stream_blocks(n), 256, 0, s>>>(F.b, r, n);
    if (int e = pmg_vcycle(P, 0, s)) return e;
    copy_kernel<<<stream_blocks(n), 256, 0, s>>>(z, F.x, n);
    return CEED_OK;
  };
  if ((st = precond(w.r, w.z))) return st;
  copy_kernel<<<stream_blocks(n), 256, 0, s>>>(w.p, w.z, n);
  double rz = host_dot(w.r, w.z, n, w.part1, &w.sc->rr_out, s, &st);
  if (st) return st;
  int it = 0;
  *nonfin = 0;
  while (it < max_iter) {
    ApplyReq a = op64;
    a.x = w.p;
    a.y = w.q;
    if ((st = launch_apply(m, a, s))) return st;
    const double pq = host_dot(w.p, w.q, n, w.part1, &w.sc->rr_out, s, &st);
    if (st) return st;
    const double alpha = rz / pq;
    if (!std::isfinite(alpha)) {
      *nonfin = 1;
      break;
    }
    const int nb = red_blocks(n);
    fcg_update_kernel<<<nb, RED_THREADS, 0, s>>>(x, w.r, w.r_old, w.p, w.q, n, alpha, w.part1);
    sum_partials_kernel<<<1, RED_THREADS, 0, s>>>(w.part1, nb, &w.sc->rr_out);
    double rr = 0.0;
    CEED_CUDA_CHECK(cudaMemcpyAsync(&rr, &w.sc->rr_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CEED_CUDA_CHECK(cudaStreamSynchronize(s));
    ++it;
    if (!std::isfinite(rr)) {
      *nonfin = 1;
      break;
    }
    if (rr <= tol * tol * bb) break;
    if ((st = precond(w.r, w.z))) return st;
    const double zr = host_dot(w.z, w.r, n, w.part1, &w.sc->rr_out, s, &st);
    const double zro = host_dot(w.z, w.r_old, n, w.part1, &w.sc->rr_out, s, &st);
    if (st) return st;
    const double beta = (zr - zro) / rz;
    rz = zr;
    xpby_kernel<<<red_blocks(n), RED_THREADS, 0, s>>>(w.p, w.z, n, beta);
  }
  *iters_out = it;
  return CEED_OK;
}

}  // namespace ceedgb

using namespace ceedgb;

extern "C" size_t ceed_dot_workspace_bytes(int64_t n) { return (size_t)red_blocks(n) * sizeof(double); }

extern "C" int ceed_dot(const double *x, const double *y, int64_t n, double *out, void *work, void *stream) {
  if (!x || !y || !out || !work || n < 0) return fail(CEED_ERR_INVALID, "bad ceed_dot arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = red_blocks(n);
  dot_partial_kernel<<<nb, RED_THREADS, 0, s>>>(x, y, n, (double *)work, nullptr);
  sum_partials_kernel<<<1, RED_THREADS, 0, s>>>((const double *)work, nb, out);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

static void fill_defaults(const ceed_cg_opts *in, ceed_cg_opts *o) {
  *o = *in;
  if (o->max_iter <= 0) o->max_iter = 10000;
  if (o->max_outer <= 0) o->max_outer = 50;
  if (o->check_every <= 0) o->check_every = 10;
  if (o->tol <= 0) o->tol = 1e-10;
  if (o->inner_tol <= 0) o->inner_tol = 1e-4;
  if (o->reliable_delta == 0.0) o->reliable_delta = 0.1;
}

extern "C" size_t ceed_cg_workspace_bytes(ceed_mesh_t m, const ceed_cg_opts *opts) {
  if (!m || !opts) return 0;
  return layout(m->n_ldof, m->E, opts->mode == CEED_CG_MIXED, nullptr, nullptr);
}

extern "C" int ceed_cg_solve(ceed_mesh_t m, const void *qdata, int prec, const double *b, double *x,
                             const ceed_cg_opts *opts_in, ceed_cg_report *report, void *work, size_t work_bytes,
                             void *stream) {
  if (int st = check_mesh(m)) return st;
  if (!qdata || !b || !x || !opts_in || !report || !work) return fail(CEED_ERR_INVALID, "null argument");
  if (m->ncomp != 1) return fail(CEED_ERR_UNSUPPORTED, "CG needs ncomp = 1");
  if (!m->has_dirichlet) return fail(CEED_ERR_INVALID, "CG needs a Dirichlet mask on the mesh");
  if (prec != CEED_F64) return fail(CEED_ERR_INVALID, "the CG operator (outer operator in MIXED mode) must be FP64");
  if (((uintptr_t)work & 255) != 0) return fail(CEED_ERR_INVALID, "workspace must be 256-byte aligned");
  ceed_cg_opts o;
  fill_defaults(opts_in, &o);
  if (o.mode != CEED_CG_FP64 && o.mode != CEED_CG_MIXED && o.mode != CEED_CG_MIXED_RELIABLE)
    return fail(CEED_ERR_INVALID, "unknown CG mode");
  const bool reliable = o.mode == CEED_CG_MIXED_RELIABLE;
  const bool mixed = o.mode == CEED_CG_MIXED || reliable;
  if (mixed && (!o.qdata_lo || (o.prec_lo != CEED_F32 && o.prec_lo != CEED_BF16 && o.prec_lo != CEED_F16 &&
                                 o.prec_lo != CEED_F32_GEO && o.prec_lo != CEED_F64_DF)))
    return fail(CEED_ERR_INVALID, "MIXED modes need qdata_lo in F32, BF16, F16, F32_GEO or F64_DF");
  if (reliable && !(o.reliable_delta > 0.0 && o.reliable_delta < 1.0))
    return fail(CEED_ERR_INVALID, "reliable_delta must lie in (0, 1)");
  if (o.op != CEED_OP_MASS && o.op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  const int64_t n = m->n_ldof;
  if (work_bytes < layout(n, m->E, mixed, nullptr, nullptr)) return fail(CEED_ERR_INVALID, "workspace too small");
  Work w;
  layout(n, m->E, mixed, (char *)work, &w);
  cudaStream_t s = (cudaStream_t)stream;
  std::memset(report, 0, sizeof(*report));

  // the two timing events are released on every return path
  struct Events {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Events() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } ev;
  CEED_CUDA_CHECK(cudaEventCreate(&ev.e0));
  CEED_CUDA_CHECK(cudaEventCreate(&ev.e1));
  cudaEvent_t ev0 = ev.e0, ev1 = ev.e1;
  CEED_CUDA_CHECK(cudaEventRecord(ev0, s));

  ApplyReq op64{};
  op64.op = o.op;
  op64.prec = CEED_F64;
  op64.qdata = qdata;
  op64.ncol = 1;
  op64.masked = 1;
  // Jacobi preconditioner from the FP64 operator
  if (int st = ceed_jacobi_diagonal(m, o.op, qdata, CEED_F64, w.dinv, CEED_APPLY_DIRICHLET, stream)) return st;
  invert_kernel<<<stream_blocks(n), 256, 0, s>>>(w.dinv, n);
  CEED_CUDA_CHECK(cudaGetLastError());

  // ||b||^2
  double bb = 0.0;
  {
    const int nb = red_blocks(n);
    dot_partial_kernel<<<nb, RED_THREADS, 0, s>>>(b, b, n, w.part1, nullptr);
    sum_partials_kernel<<<1, RED_THREADS, 0, s>>>(w.part1, nb, &w.sc->bb_out);
    CEED_CUDA_CHECK(cudaMemcpyAsync(&bb, &w.sc->bb_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  }
  if (bb == 0.0) {
    zero_kernel<<<stream_blocks(n), 256, 0, s>>>(x, n);
    CEED_CUDA_CHECK(cudaStreamSynchronize(s));
    return CEED_OK;
  }
  int status = CEED_OK;
  double rr = 0.0;
  ApplyReq oplo = op64;
  if (mixed) {
    oplo.prec = o.prec_lo;
    oplo.qdata = o.qdata_lo;
  }
  const bool fused = (o.separate_kernels == 0);
  if (reliable && o.fixed_iters <= 0) {
    if (!o.use_x0) zero_kernel<<<stream_blocks(n), 256, 0, s>>>(x, n);
    int iters = 0, evals = 0, nonfin = 0;
    double rel = 0.0;
    if (int st = reliable_run(m, op64, oplo, b, x, w, n, bb, o.tol, o.reliable_delta, o.max_iter, o.check_every, s,
                              &iters, &evals, &rel, &nonfin, fused, &report->fused))
      return st;
    report->iterations = iters;
    report->outer_iterations = evals;
    report->rel_residual = rel;
    if (nonfin) status = fail(CEED_ERR_NONFINITE, "non-finite value in a CG reduction");
    else if (!(rel <= o.tol)) status = fail(CEED_ERR_NOT_CONVERGED, "CG reached its iteration cap");
  } else if (o.fixed_iters > 0) {
    // exactly fixed_iters PCG iterations from x0 = 0 with the FP64 operator (timing runs)
    copy_kernel<<<stream_blocks(n), 256, 0, s>>>(w.r, b, n);
    int iters = 0, nonfin = 0;
    if (int st = pcg_run(m, op64, x, w, n, o.tol, o.max_iter, o.check_every, o.fixed_iters, s, &iters, &nonfin,
                         fused, &report->fused))
      return st;
    report->iterations = iters;
    report->outer_iterations = 1;
    if (nonfin) status = fail(CEED_ERR_NONFINITE, "non-finite value in a CG reduction");
    if (int st = residual(m, op64, b, x, w.q, w.r_out, n, w.part1, &w.sc->rr_out, s, &rr)) return st;
    report->rel_residual = std::sqrt(rr / bb);
  } else {
    // Refinement loop.  Each pass: true residual r = b - A64 x; stop at tol; else PCG on A d = r
    // (FP64 mode: FP64 operator, aiming at half the remaining tolerance so that the recurrence
    // residual's drift rarely forces another pass; MIXED: low-precision operator to inner_tol), x += d.
    if (!o.use_x0) zero_kernel<<<stream_blocks(n), 256, 0, s>>>(x, n);
    int total = 0, outer = 0;
    while (true) {
      if (int st = residual(m, op64, b, x, w.q, w.r_out, n, w.part1, &w.sc->rr_out, s, &rr)) return st;
      report->rel_residual = std::sqrt(rr / bb);
      if (!std::isfinite(rr)) {
        status = fail(CEED_ERR_NONFINITE, "non-finite residual");
        break;
      }
      if (report->rel_residual <= o.tol) break;
      if (outer >= o.max_outer || total >= o.max_iter) {
        status = fail(CEED_ERR_NOT_CONVERGED, "CG reached its iteration cap");
        break;
      }
      copy_kernel<<<stream_blocks(n), 256, 0, s>>>(w.r, w.r_out, n);
      // no pass aims further than half of what remains to the tolerance: MIXED passes reduce by
      // inner_tol, except a last one that needs less
      const double inner = std::min(0.5, std::max(mixed ? o.inner_tol : 0.0, 0.5 * o.tol / report->rel_residual));
      int iters = 0, nonfin = 0;
      if (!mixed && o.pmg) {
        // p-multigrid-preconditioned flexible CG on A d = r_out
        if (int st = fcg_run(m, op64, (ceed_pmg_s *)o.pmg, w.d, w.r_out, w, n, inner, o.max_iter - total, s, &iters,
                             &nonfin))
          return st;
      } else if (int st = pcg_run(m, mixed ? oplo : op64, w.d, w, n, inner, o.max_iter - total, o.check_every, 0, s,
                                  &iters, &nonfin, fused, &report->fused)) {
        return st;
      }
      total += iters;
      outer += 1;
      if (nonfin) {
        status = fail(CEED_ERR_NONFINITE, "non-finite value in a CG reduction");
        break;
      }
      axpy_kernel<<<stream_blocks(n), 256, 0, s>>>(x, w.d, n);
    }
    report->iterations = total;
    report->outer_iterations = outer;
  }
  CEED_CUDA_CHECK(cudaEventRecord(ev1, s));
  CEED_CUDA_CHECK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  report->seconds = ms * 1e-3;
  return status;
}

// ---------------------------------------------------------------------------------------------
// Dot product that allocates nothing.  The per-block partial sums live in a file-scope device
// array instead of caller-provided or library-allocated memory.  Each block sums a fixed chunk of
// CEED_DOT_NOALLOC_CHUNK entries, so the grid (and therefore the rounding order) depends only on n.
namespace {
constexpr int64_t NOALLOC_CHUNK = 8192;
constexpr int NOALLOC_MAX_BLOCKS = 32768;          // 256 KiB of FP64 partial sums
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};  // device address of the scratch, per device
}  // namespace

// Present on every device that loads the library, until the process exits.
static __device__ __align__(256) double g_dot_noalloc_scratch[NOALLOC_MAX_BLOCKS];

namespace ceedgb {
__global__ void dot_chunk_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                 double *__restrict__ part) {
  __shared__ double sh[RED_THREADS];
  const int64_t base = (int64_t)blockIdx.x * NOALLOC_CHUNK;
  double a = 0.0;
  for (int k = threadIdx.x; k < NOALLOC_CHUNK; k += RED_THREADS) {
    const int64_t i = base + k;
    if (i < n) a += x[i] * y[i];
  }
  a = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}
}  // namespace ceedgb

// Host code may not use g_dot_noalloc_scratch as a pointer (that name is a host-side shadow); the
// device address is looked up once per device, with that device current, and cached.
static int noalloc_scratch(double **out) {
  int dev = 0;
  CEED_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(CEED_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dot_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_dot_noalloc_scratch)");
    g_noalloc_ptr[dev] = (double *)p;
  }
  *out = g_noalloc_ptr[dev];
  return CEED_OK;
}

extern "C" int64_t ceed_dot_noalloc_max_n(void) { return (int64_t)NOALLOC_MAX_BLOCKS * NOALLOC_CHUNK; }

extern "C" int ceed_dot_noalloc(const double *x, const double *y, int64_t n, double *out, void *stream) {
  if (!x || !y || !out || n < 0) return fail(CEED_ERR_INVALID, "bad ceed_dot_noalloc arguments");
  if (n > ceed_dot_noalloc_max_n())
    return fail(CEED_ERR_INVALID, "ceed_dot_noalloc: n = " + std::to_string(n) + " exceeds the static scratch limit of " +
                                      std::to_string(ceed_dot_noalloc_max_n()) + " entries; use ceed_dot");
  double *scratch = nullptr;
  if (int st = noalloc_scratch(&scratch)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)std::max<int64_t>(1, (n + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
  // every block writes its slot before the sum reads it: no clearing is needed between calls
  dot_chunk_kernel<<<nb, RED_THREADS, 0, s>>>(x, y, n, scratch);
  sum_partials_kernel<<<1, RED_THREADS, 0, s>>>(scratch, nb, out);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

// ---------------------------------------------------------------- p-multigrid API
static void pmg_free(ceed_pmg_s *P) {
  if (!P) return;
  for (int l = 0; l < 4; ++l)
    if (P->lv[l].sw) ceed_schwarz_destroy(P->lv[l].sw);
  for (void *a : P->allocs) cudaFree(a);
  delete P;
}

extern "C" int ceed_pmg_create(int nlevels, const ceed_mesh_t *meshes, const void *const *qdata64,
                               const void *const *qdata_lo, const ceed_pmg_opts *opts, ceed_pmg_t *out, void *stream) {
  if (!out || !meshes || !qdata64) return fail(CEED_ERR_INVALID, "null p-multigrid argument");
  *out = nullptr;
  if (nlevels < 2 || nlevels > 4) return fail(CEED_ERR_INVALID, "p-multigrid needs 2..4 levels");
  for (int l = 0; l < nlevels; ++l) {
    if (!meshes[l] || !qdata64[l]) return fail(CEED_ERR_INVALID, "null mesh or qdata in a level");
    if (!meshes[l]->has_dirichlet) return fail(CEED_ERR_INVALID, "p-multigrid levels need the Dirichlet mask");
  }
  for (int l = 0; l + 1 < nlevels; ++l)
    if (int st = check_transfer_pair(meshes[l + 1], meshes[l])) return st;
  cudaStream_t s = (cudaStream_t)stream;
  ceed_pmg_s *P = new (std::nothrow) ceed_pmg_s();
  if (!P) return fail(CEED_ERR_OOM, "host allocation");
  if (opts) P->o = *opts;
  if (P->o.smooth_degree <= 0) P->o.smooth_degree = 4;
  if (P->o.smooth_ratio <= 1.0) P->o.smooth_ratio = 10.0;
  if (P->o.eig_iters <= 0) P->o.eig_iters = 20;
  if (P->o.coarse_tol <= 0) P->o.coarse_tol = 3e-2;
  if (P->o.coarse_max_iter <= 0) P->o.coarse_max_iter = 500;
  if (P->o.smoother != 0 && P->o.smoother != 1) {
    delete P;
    return fail(CEED_ERR_INVALID, "p-multigrid smoother: 0 (Jacobi) or 1 (Schwarz)");
  }
  P->L = nlevels;
  auto dalloc = [&](size_t bytes, void **ptr) -> int {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "p-multigrid allocation");
    P->allocs.push_back(*ptr);
    return CEED_OK;
  };
  int st = CEED_OK;
  for (int l = 0; l < nlevels && !st; ++l) {
    PmgLevel &L = P->lv[l];
    L.mesh = meshes[l];
    L.n = meshes[l]->n_ldof;
    L.op.op = CEED_OP_DIFFUSION;
    const bool lo = qdata_lo && qdata_lo[l];
    L.op.prec = lo ? P->o.prec_lo : CEED_F64;
    L.op.qdata = lo ? qdata_lo[l] : qdata64[l];
    L.op.ncol = 1;
    L.op.masked = 1;
    double **vecs[6] = {&L.x, &L.b, &L.r, &L.d, &L.q, &L.dinv};
    for (double **v : vecs)
      if (!st) st = dalloc(L.n * sizeof(double), (void **)v);
    if (!st) st = ceed_jacobi_diagonal(L.mesh, CEED_OP_DIFFUSION, qdata64[l], CEED_F64, L.dinv, CEED_APPLY_DIRICHLET, stream);
    if (!st) invert_kernel<<<stream_blocks(L.n), 256, 0, s>>>(L.dinv, L.n);
    if (!st && P->o.smoother == 1 && l + 1 < nlevels) {
      st = dalloc(L.n * sizeof(double), (void **)&L.z);
      if (!st) st = ceed_schwarz_create(L.mesh, P->o.smoother_coeff, nullptr, &L.sw, stream);
    }
  }
  if (!st) st = dalloc(RED_MAX_BLOCKS * sizeof(double), (void **)&P->part);
  if (!st) st = dalloc(sizeof(double), (void **)&P->dsum);
  if (!st) {  // coarse CG workspace
    PmgLevel &C = P->lv[nlevels - 1];
    const size_t bytes = layout(C.n, C.mesh->E, false, nullptr, nullptr);
    st = dalloc(bytes, (void **)&P->cwork);
    if (!st) layout(C.n, C.mesh->E, false, P->cwork, &P->cw);
    if (!st) copy_kernel<<<stream_blocks(C.n), 256, 0, s>>>(P->cw.dinv, C.dinv, C.n);
  }
  // lambda_max of D^{-1} A for every smoothed level (power iteration on the smoothing operator)
  for (int l = 0; l + 1 < nlevels && !st; ++l) {
    PmgLevel &L = P->lv[l];
    seed_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.x, L.n);
    double lam = 1.0;
    for (int it = 0; it < P->o.eig_iters && !st; ++it) {
      const double nx = std::sqrt(host_dot(L.x, L.x, L.n, P->part, P->dsum, s, &st));
      if (st) break;
      ApplyReq a = L.op;
      a.x = L.x;
      a.y = L.q;
      st = launch_apply(L.mesh, a, s);
      if (st) break;
      if (L.sw) {   // lambda_max of M A
        st = launch_schwarz(L.sw, L.q, L.d, 1, s);
        if (st) break;
        const double nd = std::sqrt(host_dot(L.d, L.d, L.n, P->part, P->dsum, s, &st));
        lam = nd / nx;
        copy_kernel<<<stream_blocks(L.n), 256, 0, s>>>(L.x, L.d, L.n);
        scal_kernel<<<stream_blocks(L.n), 256, 0, s>>>(L.x, L.n, 1.0 / nd);
        continue;
      }
      scale_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.d, L.dinv, L.q, L.n, 1.0);
      const double nd = std::sqrt(host_dot(L.d, L.d, L.n, P->part, P->dsum, s, &st));
      lam = nd / nx;
      scale_kernel<<<red_blocks(L.n), RED_THREADS, 0, s>>>(L.x, L.dinv, L.q, L.n, 1.0 / nd);
    }
    L.lam = lam;
  }
  if (!st) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "p-multigrid setup");
  }
  if (st) {
    pmg_free(P);
    return st;
  }
  *out = P;
  return CEED_OK;
}

extern "C" int ceed_pmg_vcycle(ceed_pmg_t P, const double *r, double *z, void *stream) {
  if (!P || !r || !z) return fail(CEED_ERR_INVALID, "bad V-cycle arguments");
  cudaStream_t s = (cudaStream_t)stream;
  PmgLevel &F = P->lv[0];
  copy_kernel<<<stream_blocks(F.n), 256, 0, s>>>(F.b, r, F.n);
  if (int st = pmg_vcycle(P, 0, s)) return st;
  copy_kernel<<<stream_blocks(F.n), 256, 0, s>>>(z, F.x, F.n);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

extern "C" int ceed_pmg_prolong(ceed_pmg_t P, int level, const double *uc, double *uf, void *stream) {
  if (!P || level < 0 || level + 1 >= P->L || !uc || !uf) return fail(CEED_ERR_INVALID, "bad prolongation arguments");
  return launch_prolong(P->lv[level + 1].mesh, P->lv[level].mesh, uc, uf, 0, (cudaStream_t)stream);
}

extern "C" int ceed_pmg_restrict(ceed_pmg_t P, int level, const double *rf, double *rc, void *stream) {
  if (!P || level < 0 || level + 1 >= P->L || !rf || !rc) return fail(CEED_ERR_INVALID, "bad restriction arguments");
  return launch_restrict(P->lv[level + 1].mesh, P->lv[level].mesh, rf, rc, (cudaStream_t)stream);
}

extern "C" int ceed_pmg_info(ceed_pmg_t P, int level, double *lambda_max) {
  if (!P || level < 0 || level >= P->L) return fail(CEED_ERR_INVALID, "bad level");
  if (lambda_max) *lambda_max = P->lv[level].lam;
  return CEED_OK;
}

extern "C" int ceed_pmg_destroy(ceed_pmg_t P) {
  if (!P) return CEED_OK;
  cudaDeviceSynchronize();
  pmg_free(P);
  return CEED_OK;
}
