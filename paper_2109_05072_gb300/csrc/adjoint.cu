// Diffusion with a per-quadrature-point coefficient k and its adjoint (collocated GLL quadrature).
//
// A(k) = sum_e P_e^T D^T G^e(k) D P_e (paper Section 2's factored form) with G_q = k_q Ghat_q,
// Ghat_q = w_q adj(J) adj(J)^T / det J, either read from stored FP64 geometry or recomputed from
// the element's 8 vertices at every point.  For L = 0.5 ||A(k) x - b||^2 and r = A(k) x - b:
//   dL/dx = A(k) r,   dL/dk_{e,q} = (grad_xi r)_q^T Ghat_q (grad_xi x)_q,
// both from one fused pass over the elements (gather x and r, three derivative passes on each,
// the pointwise products, transposed passes on k Ghat grad r, atomic-free scatter).
#include <algorithm>

#include "geometry.cuh"
#include "internal.h"

namespace ceedgb {

struct KArgs {
  const uint32_t *emap;
  const int32_t *perm;
  const double *vert;   // colour-sorted [E][8][3]
  const double *geo;    // colour-sorted [E][6][nq] or null (recompute)
  const double *k;      // caller order [E][nq]
  const double *x;
  const double *r;      // adjoint only
  double *y;            // A(k) x, or dL/dx = A(k) r
  double *dLdk;         // adjoint only, caller order
  int64_t e_begin, e_count;
  int masked;
  QRule rule;
  OpTab<double> tab;
};

template <int P, bool ADJ>
__global__ void __launch_bounds__(P * P * (P * P >= 128 ? 1 : 128 / (P * P))) kop_kernel(const KArgs a) {
  constexpr int NE = (P * P >= 128) ? 1 : (128 / (P * P));
  constexpr int NPT = P * P, ND = P * P * P;
  __shared__ double smem[NE][ADJ ? 3 : 2][ND];
  __shared__ double sv[NE][24];
  const int tid = threadIdx.x;
  const int el = tid / NPT;
  const int ij = tid - el * NPT;
  const int i = ij % P, j = ij / P;
  const int64_t e = a.e_begin + (int64_t)blockIdx.x * NE + el;
  const bool active = e < a.e_begin + a.e_count;
  double *s0 = smem[el][0], *s1 = smem[el][1];
  double *s2 = smem[el][ADJ ? 2 : 1];
  if (!a.geo)
    for (int t = ij; t < 24; t += NPT) sv[el][t] = active ? a.vert[e * 24 + t] : 0.0;

  uint32_t idx[P];
  double u[P], rv[P];
#pragma unroll
  for (int c = 0; c < P; ++c) {
    idx[c] = active ? __ldg(a.emap + e * ND + (c * P + j) * P + i) : 0u;
    const bool dir = a.masked && (idx[c] & FLAG_DIR);
    const int64_t dof = idx[c] & DOF_MASK;
    u[c] = (active && !dir) ? a.x[dof] : 0.0;
    rv[c] = (ADJ && active && !dir) ? a.r[dof] : 0.0;
  }
#pragma unroll
  for (int c = 0; c < P; ++c) {
    s0[(c * P + j) * P + i] = u[c];
    if (ADJ) s2[(c * P + j) * P + i] = rv[c];
  }
  __syncthreads();
  const double *D = a.tab.D;
  double xr[P], xs[P], xt[P];
  double gr_[P], gs_[P], gt_[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    double p0 = 0, p1 = 0, p2 = 0, q0 = 0, q1 = 0, q2 = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      p0 += D[i * P + m] * s0[(k * P + j) * P + m];
      p1 += D[j * P + m] * s0[(k * P + m) * P + i];
      p2 += D[k * P + m] * u[m];
      if (ADJ) {
        q0 += D[i * P + m] * s2[(k * P + j) * P + m];
        q1 += D[j * P + m] * s2[(k * P + m) * P + i];
        q2 += D[k * P + m] * rv[m];
      }
    }
    xr[k] = p0; xs[k] = p1; xt[k] = p2;
    gr_[k] = q0; gs_[k] = q1; gt_[k] = q2;
  }
  // pointwise: the operand of the transposed passes is k Ghat grad(w), w = x (forward) or r (adjoint)
  const int nq = ND;
  const int64_t eo = active ? a.perm[e] : 0;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int q = (k * P + j) * P + i;
    double g[6] = {0, 0, 0, 0, 0, 0};
    double kq = 0.0;
    if (active) {
      if (a.geo) {
        const double *gp = a.geo + e * 6 * nq + q;
#pragma unroll
        for (int c = 0; c < 6; ++c) g[c] = gp[c * nq];
      } else {
        double X[3], J[3][3], A[3][3];
        trilinear_map(sv[el], a.rule.x[i], a.rule.x[j], a.rule.x[k], X, J);
        const double det = adjugate(J, A);
        const double f = a.rule.w[i] * a.rule.w[j] * a.rule.w[k] / det;
        g[0] = f * (A[0][0] * A[0][0] + A[0][1] * A[0][1] + A[0][2] * A[0][2]);
        g[1] = f * (A[0][0] * A[1][0] + A[0][1] * A[1][1] + A[0][2] * A[1][2]);
        g[2] = f * (A[0][0] * A[2][0] + A[0][1] * A[2][1] + A[0][2] * A[2][2]);
        g[3] = f * (A[1][0] * A[1][0] + A[1][1] * A[1][1] + A[1][2] * A[1][2]);
        g[4] = f * (A[1][0] * A[2][0] + A[1][1] * A[2][1] + A[1][2] * A[2][2]);
        g[5] = f * (A[2][0] * A[2][0] + A[2][1] * A[2][1] + A[2][2] * A[2][2]);
      }
      kq = a.k[eo * nq + q];
    }
    const double wr = ADJ ? gr_[k] : xr[k], ws = ADJ ? gs_[k] : xs[k], wt = ADJ ? gt_[k] : xt[k];
    const double hr = g[0] * wr + g[1] * ws + g[2] * wt;
    const double hs = g[1] * wr + g[3] * ws + g[4] * wt;
    const double ht = g[2] * wr + g[4] * ws + g[5] * wt;
    if (ADJ && active) a.dLdk[eo * nq + q] = hr * xr[k] + hs * xs[k] + ht * xt[k];
    xr[k] = kq * hr;
    xs[k] = kq * hs;
    xt[k] = kq * ht;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < P; ++k) {
    s0[(k * P + j) * P + i] = xr[k];
    s1[(k * P + j) * P + i] = xs[k];
  }
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      acc += D[m * P + i] * s0[(c * P + j) * P + m];
      acc += D[m * P + j] * s1[(c * P + m) * P + i];
      acc += D[m * P + c] * xt[m];
    }
    const uint32_t v = idx[c];
    const int64_t dof = v & DOF_MASK;
    if (a.masked && (v & FLAG_DIR)) {
      if (v & FLAG_FIRST) a.y[dof] = ADJ ? a.r[dof] : a.x[dof];
    } else if (v & FLAG_FIRST) {
      a.y[dof] = acc;
    } else {
      a.y[dof] += acc;
    }
  }
}

template <int P, bool ADJ>
static int run_kop(ceed_mesh_t m, KArgs a, cudaStream_t s) {
  constexpr int NE = (P * P >= 128) ? 1 : (128 / (P * P));
  for (int c = 0; c < m->n_colors; ++c) {
    a.e_begin = m->color_start[c];
    a.e_count = m->color_start[c + 1] - a.e_begin;
    if (a.e_count == 0) continue;
    kop_kernel<P, ADJ><<<(unsigned)((a.e_count + NE - 1) / NE), P * P * NE, 0, s>>>(a);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

template <bool ADJ>
static int dispatch_kop(ceed_mesh_t m, const KArgs &a, cudaStream_t s) {
  switch (m->P) {
    case 2: return run_kop<2, ADJ>(m, a, s);
    case 3: return run_kop<3, ADJ>(m, a, s);
    case 4: return run_kop<4, ADJ>(m, a, s);
    case 5: return run_kop<5, ADJ>(m, a, s);
    case 6: return run_kop<6, ADJ>(m, a, s);
    case 7: return run_kop<7, ADJ>(m, a, s);
    case 8: return run_kop<8, ADJ>(m, a, s);
    case 9: return run_kop<9, ADJ>(m, a, s);
    default: return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
  }
}

}  // namespace ceedgb

using namespace ceedgb;

static int kop_prepare(ceed_mesh_t m, const double *k, const void *geo, KArgs *a) {
  if (int st = check_mesh(m)) return st;
  if (m->Q != m->P) return fail(CEED_ERR_UNSUPPORTED, "per-point coefficient operators need collocated GLL quadrature");
  if (m->ncomp != 1) return fail(CEED_ERR_UNSUPPORTED, "per-point coefficient operators need ncomp = 1");
  if (!k) return fail(CEED_ERR_INVALID, "null k");
  *a = KArgs{};
  a->emap = m->d_emap;
  a->perm = m->d_perm;
  a->vert = m->d_vertices;
  a->geo = (const double *)geo;
  a->k = k;
  a->rule = m->rule;
  a->tab = m->tab64;
  return CEED_OK;
}

extern "C" int ceed_apply_diffusion_k(ceed_mesh_t m, const double *k, const void *geo, const double *x, double *y,
                                      unsigned flags, void *stream) {
  KArgs a;
  if (int st = kop_prepare(m, k, geo, &a)) return st;
  if (!x || !y || x == y) return fail(CEED_ERR_INVALID, "bad x or y");
  a.x = x;
  a.y = y;
  a.masked = (flags & CEED_APPLY_DIRICHLET) ? 1 : 0;
  if (a.masked && !m->has_dirichlet) return fail(CEED_ERR_INVALID, "mesh has no Dirichlet mask");
  return dispatch_kop<false>(m, a, (cudaStream_t)stream);
}

extern "C" int ceed_apply_diffusion_adjoint(ceed_mesh_t m, const double *k, const void *geo, const double *x,
                                            const double *r, double *dLdx, double *dLdk, void *stream) {
  KArgs a;
  if (int st = kop_prepare(m, k, geo, &a)) return st;
  if (!x || !r || !dLdx || !dLdk || dLdx == r || dLdx == x) return fail(CEED_ERR_INVALID, "bad adjoint arguments");
  a.x = x;
  a.r = r;
  a.y = dLdx;
  a.dLdk = dLdk;
  a.masked = 0;
  return dispatch_kop<true>(m, a, (cudaStream_t)stream);
}
