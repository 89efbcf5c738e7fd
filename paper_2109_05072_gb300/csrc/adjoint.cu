// Diffusion with a per-quadrature-point coefficient k and its adjoint (collocated GLL quadrature).
//
// A(k) = sum_e P_e^T D^T G^e(k) D P_e (paper Section 2's factored form) with G_q = k_q Ghat_q,
// Ghat_q = w_q adj(J) adj(J)^T / det J, read from stored FP64 geometry or recomputed at every point
// from the trilinear map.  For L = 0.5 ||A(k) x - b||^2 and r = A(k) x - b:
//   dL/dx = A(k) r,   dL/dk_{e,q} = (grad_xi r)_q^T Ghat_q (grad_xi x)_q,
// both from one fused pass over the elements: gather x and r, the three derivative passes on each
// (line owners, even-odd 1D operators, padded shared tiles -- the same scheme as the apply kernel),
// the pointwise products, transposed passes on k Ghat grad r, and the atomic-free colour scatter.
// Geometry recomputation: x = a0 + a1 r + a2 s + a3 t + a4 rs + a5 rt + a6 st + a7 rst per element, so
// along a thread's column of points only t varies and J costs 6 FMAs per point (coefficients from the
// 8 vertices once per element, in shared memory).
#include <algorithm>

#include "apply_kernel.cuh"
#include "geometry.cuh"

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
  int64_t gstride;      // stored geometry per element (doubles)
  int masked;
  QRule rule;
  OpTab<double> tab;
};

template <int P>
constexpr int kop_ne() {
  return (P * P >= 128) ? 1 : (128 / (P * P));
}

template <int P, bool ADJ>
constexpr size_t kop_elem_smem() {
  return ((size_t)(ADJ ? 5 : 3) * tile_words<P>() * sizeof(double) + 24 * sizeof(double) + 127) & ~(size_t)127;
}

template <int P, bool ADJ>
__global__ void __launch_bounds__(P * P * kop_ne<P>()) kop_kernel(const KArgs a) {
  constexpr int NE = kop_ne<P>();
  constexpr int NPT = P * P, ND = P * P * P;
  constexpr int TW = tile_words<P>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int el = tid / NPT;
  const int ij = tid - el * NPT;
  const int i = ij % P, j = ij / P;
  const int64_t e = a.e_begin + (int64_t)blockIdx.x * NE + el;
  const bool active = e < a.e_begin + a.e_count;
  double *t0 = (double *)(smem_raw + el * kop_elem_smem<P, ADJ>());
  double *t1 = t0 + TW, *t2 = t1 + TW;
  double *t3 = t2 + TW, *t4 = t3 + TW;  // adjoint only
  double *coef = t0 + (ADJ ? 5 : 3) * TW;  // a1..a7 (21 values)

  if (!a.geo)  // trilinear-map coefficients of this element
    for (int t = ij; t < 21; t += NPT) {
    double v = 0.0;
    if (active) {
      const int n = t / 3, c = t % 3;  // coefficient a_{n+1}, coordinate c
      const double *V = a.vert + e * 24;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const double sr = (w & 1) ? 1.0 : -1.0, ss = (w & 2) ? 1.0 : -1.0, st = (w & 4) ? 1.0 : -1.0;
        const double sg[7] = {sr, ss, st, sr * ss, sr * st, ss * st, sr * ss * st};
        v += 0.125 * sg[n] * V[w * 3 + c];
      }
    }
    coef[t] = v;
  }

  uint32_t idx[P];
  double u[P], rv[P];
#pragma unroll
  for (int c = 0; c < P; ++c) {
    idx[c] = active ? __ldg(a.emap + e * ND + (c * P + j) * P + i) : 0u;
    const bool dir = a.masked && (idx[c] & FLAG_DIR);
    const int64_t dof = idx[c] & DOF_MASK;
    u[c] = (active && !dir) ? __ldg(a.x + dof) : 0.0;
    rv[c] = (ADJ && active && !dir) ? __ldg(a.r + dof) : 0.0;
  }
  // grad_xi x: t in registers, r and s by line owners
  double xt[P], xr[P], xs[P];
  eo_apply<P, P, -1>(a.tab.eD, u, xt);
#pragma unroll
  for (int k = 0; k < P; ++k) t0[tix<P>(k, j, i)] = u[k];
  __syncthreads();
  {
    double v[P], g[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, i, m)];
    eo_apply<P, P, -1>(a.tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t1[tix<P>(j, i, n)] = g[n];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, m, i)];
    eo_apply<P, P, -1>(a.tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t2[tix<P>(j, n, i)] = g[n];
  }
  __syncthreads();
  double rt[P];
  if constexpr (ADJ) {  // grad_xi r, the same way
    eo_apply<P, P, -1>(a.tab.eD, rv, rt);
#pragma unroll
    for (int k = 0; k < P; ++k) t0[tix<P>(k, j, i)] = rv[k];
    __syncthreads();
    double v[P], g[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, i, m)];
    eo_apply<P, P, -1>(a.tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t3[tix<P>(j, i, n)] = g[n];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, m, i)];
    eo_apply<P, P, -1>(a.tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t4[tix<P>(j, n, i)] = g[n];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    xr[k] = t1[tix<P>(k, j, i)];
    xs[k] = t2[tix<P>(k, j, i)];
  }

  // pointwise: dL/dk (adjoint) and v = k Ghat grad(w), w = x (forward) or r (adjoint)
  const int64_t eo = active ? a.perm[e] : 0;
  double c1[3], c1t[3], c2[3], c2t[3], c3[3];
  if (!a.geo) {
    const double xr0 = a.rule.x[i], xs0 = a.rule.x[j];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double a1 = coef[c], a2 = coef[3 + c], a3 = coef[6 + c], a4 = coef[9 + c];
      const double a5 = coef[12 + c], a6 = coef[15 + c], a7 = coef[18 + c];
      c1[c] = a1 + a4 * xs0;
      c1t[c] = a5 + a7 * xs0;
      c2[c] = a2 + a4 * xr0;
      c2t[c] = a6 + a7 * xr0;
      c3[c] = a3 + a5 * xr0 + a6 * xs0 + a7 * xr0 * xs0;
    }
  }
  double vt[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int q = (k * P + j) * P + i;
    double g0 = 0, g1 = 0, g2 = 0, g3 = 0, g4 = 0, g5 = 0, kq = 0;
    if (active) {
      if (a.geo) {
        const double *gp = a.geo + e * a.gstride + q;
        g0 = __ldg(gp);
        g1 = __ldg(gp + ND);
        g2 = __ldg(gp + 2 * ND);
        g3 = __ldg(gp + 3 * ND);
        g4 = __ldg(gp + 4 * ND);
        g5 = __ldg(gp + 5 * ND);
      } else {
        const double zt = a.rule.x[k];
        double J[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          J[c][0] = c1[c] + c1t[c] * zt;
          J[c][1] = c2[c] + c2t[c] * zt;
          J[c][2] = c3[c];
        }
        double A[3][3];
        const double det = adjugate(J, A);
        const double f = a.rule.w[i] * a.rule.w[j] * a.rule.w[k] / det;
        g0 = f * (A[0][0] * A[0][0] + A[0][1] * A[0][1] + A[0][2] * A[0][2]);
        g1 = f * (A[0][0] * A[1][0] + A[0][1] * A[1][1] + A[0][2] * A[1][2]);
        g2 = f * (A[0][0] * A[2][0] + A[0][1] * A[2][1] + A[0][2] * A[2][2]);
        g3 = f * (A[1][0] * A[1][0] + A[1][1] * A[1][1] + A[1][2] * A[1][2]);
        g4 = f * (A[1][0] * A[2][0] + A[1][1] * A[2][1] + A[1][2] * A[2][2]);
        g5 = f * (A[2][0] * A[2][0] + A[2][1] * A[2][1] + A[2][2] * A[2][2]);
      }
      kq = __ldg(a.k + eo * ND + q);
    }
    double wr, ws, wt;
    if constexpr (ADJ) {
      wr = t3[tix<P>(k, j, i)];
      ws = t4[tix<P>(k, j, i)];
      wt = rt[k];
    } else {
      wr = xr[k];
      ws = xs[k];
      wt = xt[k];
    }
    const double hr = g0 * wr + g1 * ws + g2 * wt;
    const double hs = g1 * wr + g3 * ws + g4 * wt;
    const double ht = g2 * wr + g4 * ws + g5 * wt;
    if (ADJ && active) a.dLdk[eo * ND + q] = hr * xr[k] + hs * xs[k] + ht * xt[k];
    t1[tix<P>(k, j, i)] = kq * hr;
    t2[tix<P>(k, j, i)] = kq * hs;
    vt[k] = kq * ht;
  }
  __syncthreads();
  {  // transposed passes
    double v[P], g[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t1[tix<P>(j, i, m)];
    eo_apply<P, P, -1>(a.tab.eDT, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t0[tix<P>(j, i, n)] = g[n];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t2[tix<P>(j, m, i)];
    eo_apply<P, P, -1>(a.tab.eDT, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t2[tix<P>(j, n, i)] = g[n];
  }
  double yt[P];
  eo_apply<P, P, -1>(a.tab.eDT, vt, yt);
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    const double acc = yt[c] + t0[tix<P>(c, j, i)] + t2[tix<P>(c, j, i)];
    const uint32_t v = idx[c];
    const int64_t dof = v & DOF_MASK;
    if (a.masked && (v & FLAG_DIR)) {
      if (v & FLAG_FIRST) a.y[dof] = ADJ ? a.r[dof] : a.x[dof];
    } else if (v & FLAG_FIRST) {
      a.y[dof] = acc;
    } else {
      a.y[dof] = __ldcg(a.y + dof) + acc;
    }
  }
}

// The same operator and adjoint with FP64 accuracy on the FP32 pipe (flag CEED_APPLY_F64_DF): values
// as double-float pairs (split from FP64 on the gather, collapsed to FP64 on the scatter), every
// contraction, the pointwise products and the dL/dk bilinear form as compensated dot products
// (Dot2, df.cuh); the geometry is the stored FP64 form, split per point.
template <int P, bool ADJ>
__global__ void __launch_bounds__(P * P * kop_ne<P>()) kop_df_kernel(const KArgs a, const OpTab<DF> tab) {
  constexpr int NE = kop_ne<P>();
  constexpr int NPT = P * P, ND = P * P * P;
  constexpr int TW = tile_words<P>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int el = tid / NPT;
  const int ij = tid - el * NPT;
  const int i = ij % P, j = ij / P;
  const int64_t e = a.e_begin + (int64_t)blockIdx.x * NE + el;
  const bool active = e < a.e_begin + a.e_count;
  DF *t0 = (DF *)(smem_raw + el * kop_elem_smem<P, ADJ>());
  DF *t1 = t0 + TW, *t2 = t1 + TW;
  DF *t3 = t2 + TW, *t4 = t3 + TW;  // adjoint only

  uint32_t idx[P];
  DF u[P], rv[P];
#pragma unroll
  for (int c = 0; c < P; ++c) {
    idx[c] = active ? __ldg(a.emap + e * ND + (c * P + j) * P + i) : 0u;
    const bool dir = a.masked && (idx[c] & FLAG_DIR);
    const int64_t dof = idx[c] & DOF_MASK;
    u[c] = (active && !dir) ? LVec<DF>::in(__ldg(a.x + dof)) : DF(0.f, 0.f);
    rv[c] = (ADJ && active && !dir) ? LVec<DF>::in(__ldg(a.r + dof)) : DF(0.f, 0.f);
  }
  DF xt[P], xr[P], xs[P];
  eo_apply<P, P, -1>(tab.eD, u, xt);
#pragma unroll
  for (int k = 0; k < P; ++k) t0[tix<P>(k, j, i)] = u[k];
  __syncthreads();
  {
    DF v[P], g[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, i, m)];
    eo_apply<P, P, -1>(tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t1[tix<P>(j, i, n)] = g[n];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, m, i)];
    eo_apply<P, P, -1>(tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t2[tix<P>(j, n, i)] = g[n];
  }
  __syncthreads();
  DF rt[P];
  if constexpr (ADJ) {
    eo_apply<P, P, -1>(tab.eD, rv, rt);
#pragma unroll
    for (int k = 0; k < P; ++k) t0[tix<P>(k, j, i)] = rv[k];
    __syncthreads();
    DF v[P], g[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, i, m)];
    eo_apply<P, P, -1>(tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t3[tix<P>(j, i, n)] = g[n];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t0[tix<P>(j, m, i)];
    eo_apply<P, P, -1>(tab.eD, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t4[tix<P>(j, n, i)] = g[n];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    xr[k] = t1[tix<P>(k, j, i)];
    xs[k] = t2[tix<P>(k, j, i)];
  }
  const int64_t eo = active ? a.perm[e] : 0;
  DF vt[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int q = (k * P + j) * P + i;
    DF g0(0.f, 0.f), g1(0.f, 0.f), g2(0.f, 0.f), g3(0.f, 0.f), g4(0.f, 0.f), g5(0.f, 0.f), kq(0.f, 0.f);
    if (active) {
      const double *gp = a.geo + e * a.gstride + q;
      g0 = LVec<DF>::in(__ldg(gp));
      g1 = LVec<DF>::in(__ldg(gp + ND));
      g2 = LVec<DF>::in(__ldg(gp + 2 * ND));
      g3 = LVec<DF>::in(__ldg(gp + 3 * ND));
      g4 = LVec<DF>::in(__ldg(gp + 4 * ND));
      g5 = LVec<DF>::in(__ldg(gp + 5 * ND));
      kq = LVec<DF>::in(__ldg(a.k + eo * ND + q));
    }
    DF wr, ws, wt;
    if constexpr (ADJ) {
      wr = t3[tix<P>(k, j, i)];
      ws = t4[tix<P>(k, j, i)];
      wt = rt[k];
    } else {
      wr = xr[k];
      ws = xs[k];
      wt = xt[k];
    }
    const DF hr = dot3<DF>(g0, wr, g1, ws, g2, wt);
    const DF hs = dot3<DF>(g1, wr, g3, ws, g4, wt);
    const DF ht = dot3<DF>(g2, wr, g4, ws, g5, wt);
    if (ADJ && active) a.dLdk[eo * ND + q] = LVec<DF>::out(dot3<DF>(hr, xr[k], hs, xs[k], ht, xt[k]));
    t1[tix<P>(k, j, i)] = qmul<DF>(kq, hr);
    t2[tix<P>(k, j, i)] = qmul<DF>(kq, hs);
    vt[k] = qmul<DF>(kq, ht);
  }
  __syncthreads();
  {  // transposed passes
    DF v[P], g[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t1[tix<P>(j, i, m)];
    eo_apply<P, P, -1>(tab.eDT, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t0[tix<P>(j, i, n)] = g[n];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = t2[tix<P>(j, m, i)];
    eo_apply<P, P, -1>(tab.eDT, v, g);
#pragma unroll
    for (int n = 0; n < P; ++n) t2[tix<P>(j, n, i)] = g[n];
  }
  DF yt[P];
  eo_apply<P, P, -1>(tab.eDT, vt, yt);
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    const DF acc = add3<DF>(yt[c], t0[tix<P>(c, j, i)], t2[tix<P>(c, j, i)]);
    const uint32_t v = idx[c];
    const int64_t dof = v & DOF_MASK;
    if (a.masked && (v & FLAG_DIR)) {
      if (v & FLAG_FIRST) a.y[dof] = ADJ ? a.r[dof] : a.x[dof];
    } else if (v & FLAG_FIRST) {
      a.y[dof] = LVec<DF>::out(acc);
    } else {
      a.y[dof] = LVec<DF>::add(__ldcg(a.y + dof), acc);
    }
  }
}

template <int P, bool ADJ>
static int run_kop_df(ceed_mesh_t m, KArgs a, cudaStream_t s) {
  constexpr int NE = kop_ne<P>();
  const size_t smem = NE * kop_elem_smem<P, ADJ>();
  if (int st = ensure_dynamic_smem((const void *)kop_df_kernel<P, ADJ>, smem)) return st;
  for (int c = 0; c < m->n_colors; ++c) {
    a.e_begin = m->color_start[c];
    a.e_count = m->color_start[c + 1] - a.e_begin;
    if (a.e_count == 0) continue;
    kop_df_kernel<P, ADJ><<<(unsigned)((a.e_count + NE - 1) / NE), P * P * NE, smem, s>>>(a, m->tabdf);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

template <int P, bool ADJ>
static int run_kop(ceed_mesh_t m, KArgs a, cudaStream_t s) {
  constexpr int NE = kop_ne<P>();
  const size_t smem = NE * kop_elem_smem<P, ADJ>();
  if (int st = ensure_dynamic_smem((const void *)kop_kernel<P, ADJ>, smem)) return st;
  for (int c = 0; c < m->n_colors; ++c) {
    a.e_begin = m->color_start[c];
    a.e_count = m->color_start[c + 1] - a.e_begin;
    if (a.e_count == 0) continue;
    kop_kernel<P, ADJ><<<(unsigned)((a.e_count + NE - 1) / NE), P * P * NE, smem, s>>>(a);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

template <bool ADJ>
static int dispatch_kop(ceed_mesh_t m, const KArgs &a, bool df, cudaStream_t s) {
  if (df) {
    switch (m->P) {
      case 2: return run_kop_df<2, ADJ>(m, a, s);
      case 3: return run_kop_df<3, ADJ>(m, a, s);
      case 4: return run_kop_df<4, ADJ>(m, a, s);
      case 5: return run_kop_df<5, ADJ>(m, a, s);
      case 6: return run_kop_df<6, ADJ>(m, a, s);
      case 7: return run_kop_df<7, ADJ>(m, a, s);
      case 8: return run_kop_df<8, ADJ>(m, a, s);
      case 9: return run_kop_df<9, ADJ>(m, a, s);
      default: return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
    }
  }
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
  if (!geo && m->d_coords)
    return fail(CEED_ERR_UNSUPPORTED, "recomputed geometry is the trilinear map; pass stored geometry for a curved mesh");
  *a = KArgs{};
  a->emap = m->d_emap;
  a->perm = m->d_perm;
  a->vert = m->d_vertices;
  a->geo = (const double *)geo;
  a->gstride = qdata_estride(CEED_OP_DIFFUSION, 8, m->Q);
  a->k = k;
  a->rule = m->rule;
  a->tab = m->tab64;
  return CEED_OK;
}

// the arithmetic requested by the flags: CEED_APPLY_F64_DF needs the stored geometry
static int kop_df_flag(const void *geo, unsigned flags, bool *df) {
  if (flags & ~(CEED_APPLY_DIRICHLET | CEED_APPLY_F64_DF)) return fail(CEED_ERR_INVALID, "unknown flag bits");
  *df = (flags & CEED_APPLY_F64_DF) != 0;
  if (*df && !geo) return fail(CEED_ERR_UNSUPPORTED, "CEED_APPLY_F64_DF needs the stored geometry");
  return CEED_OK;
}

extern "C" int ceed_apply_diffusion_k(ceed_mesh_t m, const double *k, const void *geo, const double *x, double *y,
                                      unsigned flags, void *stream) {
  KArgs a;
  if (int st = kop_prepare(m, k, geo, &a)) return st;
  if (!x || !y || x == y) return fail(CEED_ERR_INVALID, "bad x or y");
  bool df = false;
  if (int st = kop_df_flag(geo, flags, &df)) return st;
  a.x = x;
  a.y = y;
  a.masked = (flags & CEED_APPLY_DIRICHLET) ? 1 : 0;
  if (a.masked && !m->has_dirichlet) return fail(CEED_ERR_INVALID, "mesh has no Dirichlet mask");
  return dispatch_kop<false>(m, a, df, (cudaStream_t)stream);
}

extern "C" int ceed_apply_diffusion_adjoint(ceed_mesh_t m, const double *k, const void *geo, const double *x,
                                            const double *r, double *dLdx, double *dLdk, unsigned flags,
                                            void *stream) {
  KArgs a;
  if (int st = kop_prepare(m, k, geo, &a)) return st;
  if (!x || !r || !dLdx || !dLdk || dLdx == r || dLdx == x) return fail(CEED_ERR_INVALID, "bad adjoint arguments");
  if (flags & CEED_APPLY_DIRICHLET) return fail(CEED_ERR_INVALID, "the adjoint is unmasked");
  bool df = false;
  if (int st = kop_df_flag(geo, flags, &df)) return st;
  a.x = x;
  a.r = r;
  a.y = dLdx;
  a.dLdk = dLdk;
  a.masked = 0;
  return dispatch_kop<true>(m, a, df, (cudaStream_t)stream);
}
