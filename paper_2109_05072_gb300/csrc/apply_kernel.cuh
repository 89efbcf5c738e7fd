// Fused matrix-free element kernel: gather (L->E), sum-factorized 1D contractions to the
// quadrature points, pointwise quadrature operator, transposed contractions, scatter-add (E->L).
//
// Paper Section 2: w_L = A_L u_L with A_L = block-diag(A^e), A^e = D^T G^e D; the 3D derivative
// is applied as 1D contractions u_r(r_i, s_j, t_k) = sum_m Dhat_im u_mjk (and likewise along s, t),
// and G^e is six diagonal matrices G_rr ... G_tt.  Section 3 (cuda-gen): the whole operator in one
// kernel with no global temporaries.  Section 1: sum factorization, O(p^{d+1}) work per element.
//
// Thread layout: Q x Q threads per element, thread (i, j) owns the column of points (i, j, 0..Q-1)
// in registers; planes are exchanged through shared memory for the r and s passes, the t pass
// stays in registers.  NE elements per thread block.  Elements of one colour share no node, so
// the scatter is a plain (non-atomic) store for the first writer of a node and a load-add-store
// for later colours: deterministic and atomic-free.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace ceedgb {

__device__ __forceinline__ double ld_q(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_q(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_q(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld_q(const __half *p) { return __half2float(__ldg(p)); }

template <int Q>
constexpr int elems_per_block() {
  return (Q * Q >= 128) ? 1 : (128 / (Q * Q));
}

template <int P, int Q, int OP, typename T, typename TQ>
__global__ void __launch_bounds__(Q * Q * elems_per_block<Q>())
apply_kernel(const uint32_t *__restrict__ emap, const TQ *__restrict__ qdata, const double *__restrict__ x,
             double *__restrict__ y, int64_t e_begin, int64_t e_count, int ncol, int masked, const OpTab<T> tab) {
  constexpr int NE = elems_per_block<Q>();
  constexpr int NPT = Q * Q;
  constexpr bool COLLOC = (P == Q);
  constexpr int ND = P * P * P;
  constexpr int NQ = Q * Q * Q;
  constexpr int NCQ = (OP == CEED_OP_DIFFUSION) ? 6 : 1;
  __shared__ T smem[NE][2][NQ];

  const int tid = threadIdx.x;
  const int el = tid / NPT;
  const int ij = tid - el * NPT;
  const int i = ij % Q, j = ij / Q;
  const int64_t e = e_begin + (int64_t)blockIdx.x * NE + el;
  const bool active = e < e_begin + e_count;
  const bool node_thread = (i < P) && (j < P);
  T *s0 = smem[el][0];
  T *s1 = smem[el][1];

  uint32_t idx[P];
#pragma unroll
  for (int c = 0; c < P; ++c) idx[c] = 0;
  if (active && node_thread) {
    const uint32_t *em = emap + e * ND + j * P + i;
#pragma unroll
    for (int c = 0; c < P; ++c) idx[c] = __ldg(em + c * P * P);
  }
  const TQ *qd = qdata + (active ? e : e_begin) * (int64_t)(NCQ * NQ) + ij;

  for (int col = 0; col < ncol; ++col) {
    // ---------------- gather (L -> E)
    T u[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      double xv = 0.0;
      if (active && node_thread) {
        const uint32_t v = idx[c];
        if (!(masked && (v & FLAG_DIR))) xv = __ldg(x + (int64_t)(v & DOF_MASK) * ncol + col);
      }
      u[c] = (T)xv;
    }

    // ---------------- interpolate to the quadrature points (identity when collocated)
    T uq[Q];
    if constexpr (COLLOC) {
#pragma unroll
      for (int k = 0; k < Q; ++k) uq[k] = u[k];
    } else {
      if (node_thread) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          T a = 0;
#pragma unroll
          for (int c = 0; c < P; ++c) a += tab.B[k * P + c] * u[c];
          s0[(k * Q + j) * Q + i] = a;
        }
      }
      __syncthreads();
      if (i < P) {
        T Bj[P];
#pragma unroll
        for (int b = 0; b < P; ++b) Bj[b] = tab.B[j * P + b];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          T a = 0;
#pragma unroll
          for (int b = 0; b < P; ++b) a += Bj[b] * s0[(k * Q + b) * Q + i];
          s1[(k * Q + j) * Q + i] = a;
        }
      }
      __syncthreads();
      T Bi[P];
#pragma unroll
      for (int a = 0; a < P; ++a) Bi[a] = tab.B[i * P + a];
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        T a = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) a += Bi[m] * s1[(k * Q + j) * Q + m];
        uq[k] = a;
      }
    }

    // ---------------- quadrature-point operator
    T w[Q];
    if constexpr (OP == CEED_OP_MASS) {
#pragma unroll
      for (int k = 0; k < Q; ++k) w[k] = active ? (T)ld_q(qd + k * NPT) * uq[k] : (T)0;
    } else {
#pragma unroll
      for (int k = 0; k < Q; ++k) s0[(k * Q + j) * Q + i] = uq[k];
      __syncthreads();
      T ur[Q], us[Q], ut[Q];
      {
        T Di[Q], Dj[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) {
          Di[m] = tab.D[i * Q + m];
          Dj[m] = tab.D[j * Q + m];
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          T a = 0, b = 0, c = 0;
#pragma unroll
          for (int m = 0; m < Q; ++m) {
            a += Di[m] * s0[(k * Q + j) * Q + m];
            b += Dj[m] * s0[(k * Q + m) * Q + i];
            c += tab.D[k * Q + m] * uq[m];
          }
          ur[k] = a;
          us[k] = b;
          ut[k] = c;
        }
      }
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        T vr = 0, vs = 0, vt = 0;
        if (active) {
          const TQ *g = qd + k * NPT;
          const T grr = (T)ld_q(g), grs = (T)ld_q(g + NQ), grt = (T)ld_q(g + 2 * NQ);
          const T gss = (T)ld_q(g + 3 * NQ), gst = (T)ld_q(g + 4 * NQ), gtt = (T)ld_q(g + 5 * NQ);
          vr = grr * ur[k] + grs * us[k] + grt * ut[k];
          vs = grs * ur[k] + gss * us[k] + gst * ut[k];
          vt = grt * ur[k] + gst * us[k] + gtt * ut[k];
        }
        ur[k] = vr;
        us[k] = vs;
        ut[k] = vt;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        s0[(k * Q + j) * Q + i] = ur[k];
        s1[(k * Q + j) * Q + i] = us[k];
      }
      __syncthreads();
      T DTi[Q], DTj[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        DTi[m] = tab.D[m * Q + i];
        DTj[m] = tab.D[m * Q + j];
      }
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        T a = 0;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
          a += DTi[m] * s0[(k * Q + j) * Q + m];
          a += DTj[m] * s1[(k * Q + m) * Q + i];
          a += tab.D[m * Q + k] * ut[m];
        }
        w[k] = a;
      }
    }

    // ---------------- transposed interpolation back to the nodes
    T yv[P];
    if constexpr (COLLOC) {
#pragma unroll
      for (int c = 0; c < P; ++c) yv[c] = w[c];
    } else {
      __syncthreads();
#pragma unroll
      for (int k = 0; k < Q; ++k) s0[(k * Q + j) * Q + i] = w[k];
      __syncthreads();
      if (i < P) {
        T BTa[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) BTa[m] = tab.B[m * P + i];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          T a = 0;
#pragma unroll
          for (int m = 0; m < Q; ++m) a += BTa[m] * s0[(k * Q + j) * Q + m];
          s1[(k * Q + j) * Q + i] = a;
        }
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < P; ++c) yv[c] = 0;
      if (node_thread) {
        T BTb[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) BTb[m] = tab.B[m * P + j];
        T t[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          T a = 0;
#pragma unroll
          for (int m = 0; m < Q; ++m) a += BTb[m] * s1[(k * Q + m) * Q + i];
          t[k] = a;
        }
#pragma unroll
        for (int c = 0; c < P; ++c) {
          T a = 0;
#pragma unroll
          for (int k = 0; k < Q; ++k) a += tab.B[k * P + c] * t[k];
          yv[c] = a;
        }
      }
    }

    // ---------------- scatter-add (E -> L), atomic-free
    if (active && node_thread) {
#pragma unroll
      for (int c = 0; c < P; ++c) {
        const uint32_t v = idx[c];
        const int64_t o = (int64_t)(v & DOF_MASK) * ncol + col;
        if (masked && (v & FLAG_DIR)) {
          if (v & FLAG_FIRST) y[o] = x[o];
        } else if (v & FLAG_FIRST) {
          y[o] = (double)yv[c];
        } else {
          y[o] += (double)yv[c];
        }
      }
    }
    if (col + 1 < ncol) __syncthreads();
  }
}

// Launch one kernel per colour for a fixed (P, Q, op, T, TQ).
template <int P, int Q, int OP, typename T, typename TQ>
int launch_colours(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, cudaStream_t s) {
  constexpr int NE = elems_per_block<Q>();
  const dim3 block(Q * Q * NE);
  for (int c = 0; c < m->n_colors; ++c) {
    const int64_t b = m->color_start[c], n = m->color_start[c + 1] - b;
    if (n == 0) continue;
    const dim3 grid((unsigned)((n + NE - 1) / NE));
    apply_kernel<P, Q, OP, T, TQ><<<grid, block, 0, s>>>(m->d_emap, (const TQ *)r.qdata, r.x, r.y, b, n, r.ncol,
                                                         r.masked, tab);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

// Dispatch on (P, collocated?, op) for one (T, TQ) pair.
template <typename T, typename TQ>
int dispatch_apply(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, cudaStream_t s) {
  const bool colloc = (m->Q == m->P);
#define CEEDGB_CASE(PP)                                                                                   \
  case PP:                                                                                               \
    if (colloc)                                                                                          \
      return r.op == CEED_OP_MASS ? launch_colours<PP, PP, CEED_OP_MASS, T, TQ>(m, tab, r, s)             \
                                  : launch_colours<PP, PP, CEED_OP_DIFFUSION, T, TQ>(m, tab, r, s);      \
    else                                                                                                 \
      return r.op == CEED_OP_MASS ? launch_colours<PP, PP + 1, CEED_OP_MASS, T, TQ>(m, tab, r, s)         \
                                  : launch_colours<PP, PP + 1, CEED_OP_DIFFUSION, T, TQ>(m, tab, r, s);
  switch (m->P) {
    CEEDGB_CASE(2)
    CEEDGB_CASE(3)
    CEEDGB_CASE(4)
    CEEDGB_CASE(5)
    CEEDGB_CASE(6)
    CEEDGB_CASE(7)
    CEEDGB_CASE(8)
    CEEDGB_CASE(9)
    default:
      return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
  }
#undef CEEDGB_CASE
}

}  // namespace ceedgb
