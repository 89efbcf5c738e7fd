// Setup-time kernels: quadrature data (geometric factors), manufactured right-hand side, Jacobi diagonal.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "geometry.cuh"
#include "internal.h"

namespace ceedgb {

template <typename TQ>
__device__ __forceinline__ TQ to_store(double v);
template <>
__device__ __forceinline__ double to_store<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_store<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
template <>
__device__ __forceinline__ __half to_store<__half>(double v) { return __float2half_rn((float)v); }
template <>
__device__ __forceinline__ DF to_store<DF>(double v) { return df_from_double(v); }

// Quadrature data at one point q of sorted element s from the physical point X and J = dx/dxi.
// Paper Section 2: the symmetric geometric tensor G^e stored as six diagonal matrices; here
// G = w k adj(J) adj(J)^T / det J (= w k det J J^{-1} J^{-T}), mass w |det J| rho.
struct QdataCoeff {
  int op, coeff_kind;
  double cconst;
  const double *coeff;   // PER_QPT: [caller's element][nq]
  const int32_t *perm;   // sorted position -> caller's element
};

template <typename TQ>
__device__ __forceinline__ void qdata_point(const QdataCoeff &c, int64_t s, int q, int nq, double w, const double X[3],
                                            const double J[3][3], TQ *__restrict__ out_e, int *err) {
  double A[3][3];
  const double det = adjugate(J, A);
  if (!(det > 0.0)) *err = CEED_ERR_BAD_GEOMETRY;
  double kq = 1.0;
  if (c.coeff_kind == CEED_COEFF_CONST) kq = c.cconst;
  else if (c.coeff_kind == CEED_COEFF_SINE) kq = sine_coefficient(X);
  else if (c.coeff_kind == CEED_COEFF_PER_QPT) kq = c.coeff[(int64_t)c.perm[s] * nq + q];
  if (c.op == CEED_OP_MASS) {
    out_e[q] = to_store<TQ>(w * fabs(det) * kq);
  } else {
    const double f = w * kq / det;
    TQ *o = out_e + q;
    o[0 * nq] = to_store<TQ>(f * (A[0][0] * A[0][0] + A[0][1] * A[0][1] + A[0][2] * A[0][2]));
    o[1 * nq] = to_store<TQ>(f * (A[0][0] * A[1][0] + A[0][1] * A[1][1] + A[0][2] * A[1][2]));
    o[2 * nq] = to_store<TQ>(f * (A[0][0] * A[2][0] + A[0][1] * A[2][1] + A[0][2] * A[2][2]));
    o[3 * nq] = to_store<TQ>(f * (A[1][0] * A[1][0] + A[1][1] * A[1][1] + A[1][2] * A[1][2]));
    o[4 * nq] = to_store<TQ>(f * (A[1][0] * A[2][0] + A[1][1] * A[2][1] + A[1][2] * A[2][2]));
    o[5 * nq] = to_store<TQ>(f * (A[2][0] * A[2][0] + A[2][1] * A[2][1] + A[2][2] * A[2][2]));
  }
}

// Trilinear geometry: one thread per (colour-sorted element, quadrature point).
template <typename TQ>
__global__ void qdata_kernel(int64_t E, int Q, const double *__restrict__ vert, QdataCoeff c, QRule rule,
                             TQ *__restrict__ out, int64_t estride, int *err) {
  const int nq = Q * Q * Q;
  const int64_t total = E * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / nq;
    const int q = (int)(t - s * nq);
    const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
    double X[3], J[3][3];
    trilinear_map(vert + s * 24, rule.x[i], rule.x[j], rule.x[k], X, J);
    qdata_point<TQ>(c, s, q, nq, rule.w[i] * rule.w[j] * rule.w[k], X, J, out + s * estride, err);
  }
}

// Curved (isoparametric) geometry: one block of ISO_THREADS per colour-sorted element (grid-stride).
template <typename TQ>
__global__ void __launch_bounds__(ISO_THREADS)
iso_qdata_kernel(int64_t E, int P, int Q, const uint32_t *__restrict__ emap, const double *__restrict__ coords,
                 const IsoTab tab, QdataCoeff c, QRule rule, TQ *__restrict__ out, int64_t estride, int *err) {
  extern __shared__ double sm[];
  const int nq = Q * Q * Q, nd = P * P * P;
  for (int64_t s = blockIdx.x; s < E; s += gridDim.x) {
    double X[ISO_PPT][3], J[ISO_PPT][3][3];
    iso_geometry(coords, emap + s * nd, P, Q, tab, sm, X, J);
#pragma unroll
    for (int t = 0; t < ISO_PPT; ++t) {
      const int q = threadIdx.x + t * blockDim.x;
      if (q >= nq) continue;
      const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
      qdata_point<TQ>(c, s, q, nq, rule.w[i] * rule.w[j] * rule.w[k], X[t], J[t], out + s * estride, err);
    }
  }
}

// Node positions under the trilinear maps: one thread per (sorted element, node); first writers store.
struct NodeCoordArgs {
  const uint32_t *emap;
  const double *vert;
  double *coords;
  int64_t E;
  int P;
  double x[MAX_P];  // GLL nodes
};

__global__ void node_coords_kernel(const NodeCoordArgs a) {
  const int nd = a.P * a.P * a.P;
  const int64_t total = a.E * nd;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / nd;
    const int n = (int)(t - s * nd);
    const uint32_t v = a.emap[t];
    if (!(v & FLAG_FIRST)) continue;
    const int ia = n % a.P, ib = (n / a.P) % a.P, ic = n / (a.P * a.P);
    double X[3], J[3][3];
    trilinear_map(a.vert + s * 24, a.x[ia], a.x[ib], a.x[ic], X, J);
    double *o = a.coords + (int64_t)(v & DOF_MASK) * 3;
    o[0] = X[0];
    o[1] = X[1];
    o[2] = X[2];
  }
}

// 1D tables of the isoparametric map: B (nodal basis at the points) and G = D B (its derivative;
// exact, since D differentiates the degree Q-1 interpolant of a degree p <= Q-1 polynomial).
static IsoTab make_iso_tab(ceed_mesh_t m) {
  IsoTab t{};
  const int P = m->P, Q = m->Q;
  for (int q = 0; q < Q; ++q)
    for (int a = 0; a < P; ++a) {
      t.B[q * P + a] = m->tab64.B[q * P + a];
      double g = 0.0;
      for (int r = 0; r < Q; ++r) g += m->tab64.D[q * Q + r] * m->tab64.B[r * P + a];
      t.G[q * P + a] = g;
    }
  return t;
}

// Quadrature data for the on-the-fly-geometry FP32 diffusion operator: per element the
// coefficients a1..a7 of the trilinear map x = a0 + a1 r + a2 s + a3 t + a4 rs + a5 rt + a6 st +
// a7 rst (computed in FP64 from the 8 vertices, stored FP32), then w_q k_q at every point.
__global__ void geo_qdata_kernel(int64_t E, int Q, const double *__restrict__ vert, const int32_t *__restrict__ perm,
                                 int coeff_kind, double cconst, const double *__restrict__ coeff, QRule rule,
                                 float *__restrict__ out, int64_t estride, int *err) {
  const int nq = Q * Q * Q;
  const int64_t total = E * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / nq;
    const int q = (int)(t - s * nq);
    const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
    const double *V = vert + s * 24;
    if (q == 0) {
      for (int c = 0; c < 3; ++c) {
        double a[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int v = 0; v < 8; ++v) {
          const double sr = (v & 1) ? 1.0 : -1.0, ss = (v & 2) ? 1.0 : -1.0, st = (v & 4) ? 1.0 : -1.0;
          const double xv = 0.125 * V[v * 3 + c];
          a[0] += sr * xv;
          a[1] += ss * xv;
          a[2] += st * xv;
          a[3] += sr * ss * xv;
          a[4] += sr * st * xv;
          a[5] += ss * st * xv;
          a[6] += sr * ss * st * xv;
        }
        for (int n = 0; n < 7; ++n) out[s * estride + n * 3 + c] = (float)a[n];
      }
      for (int n = 21; n < GEO_COEFFS; ++n) out[s * estride + n] = 0.f;
    }
    double X[3], J[3][3], A[3][3];
    trilinear_map(V, rule.x[i], rule.x[j], rule.x[k], X, J);
    const double det = adjugate(J, A);
    if (!(det > 0.0)) *err = CEED_ERR_BAD_GEOMETRY;
    double kq = 1.0;
    if (coeff_kind == CEED_COEFF_CONST) kq = cconst;
    else if (coeff_kind == CEED_COEFF_SINE) kq = sine_coefficient(X);
    else if (coeff_kind == CEED_COEFF_PER_QPT) kq = coeff[(int64_t)perm[s] * nq + q];
    out[s * estride + GEO_COEFFS + q] = (float)(rule.w[i] * rule.w[j] * rule.w[k] * kq);
  }
}

// Per-element vector assembled with the same atomic-free colour scheme as the apply.
// mode 0: manufactured RHS b_i = sum_q w |det J| f(x_q) phi_i(x_q)
// mode 1: Jacobi diagonal of the mass operator, sum_q qd_q phi_i(x_q)^2
// mode 2: Jacobi diagonal of the diffusion operator, sum_q grad phi_i^T G_q grad phi_i
struct ElemVecArgs {
  const uint32_t *emap;
  const double *vert;
  const double *coords;   // curved geometry (mode 0), or null for the trilinear map
  IsoTab iso;
  const double *qd;       // FP64 qdata (modes 1, 2)
  double *out;
  int64_t e_begin, e_count;
  int P, Q, ncomp, masked, mode, coeff_kind;
  QRule rule;
  OpTab<double> tab;
};

__global__ void elemvec_kernel(ElemVecArgs a) {
  const int64_t e = a.e_begin + blockIdx.x;
  if (e >= a.e_begin + a.e_count) return;
  const int P = a.P, Q = a.Q, nd = P * P * P, nq = Q * Q * Q;
  extern __shared__ double sh[];
  double *fq = sh;           // [nq] point values (mode 0)
  double *G1 = sh + nq;      // [Q][P] derivative of the nodal basis at the points, G1 = D B (Gauss only)
  if (P != Q) {
    for (int t = threadIdx.x; t < Q * P; t += blockDim.x) {
      const int q = t / P, c = t % P;
      double s = 0.0;
      for (int m = 0; m < Q; ++m) s += a.tab.D[q * Q + m] * a.tab.B[m * P + c];
      G1[t] = s;
    }
    __syncthreads();
  }
  if (a.mode == 0 && a.coords) {  // curved geometry; blockDim.x * ISO_PPT >= nq
    double X[ISO_PPT][3], J[ISO_PPT][3][3];
    iso_geometry(a.coords, a.emap + e * nd, P, Q, a.iso, G1 + MAX_Q * MAX_P, X, J);
#pragma unroll
    for (int t = 0; t < ISO_PPT; ++t) {
      const int q = threadIdx.x + t * blockDim.x;
      if (q >= nq) continue;
      const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
      double A[3][3];
      const double det = adjugate(J[t], A);
      fq[q] = a.rule.w[i] * a.rule.w[j] * a.rule.w[k] * fabs(det) * manufactured_source(X[t], a.coeff_kind);
    }
    __syncthreads();
  } else if (a.mode == 0) {
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
      double X[3], J[3][3], A[3][3];
      trilinear_map(a.vert + e * 24, a.rule.x[i], a.rule.x[j], a.rule.x[k], X, J);
      const double det = adjugate(J, A);
      fq[q] = a.rule.w[i] * a.rule.w[j] * a.rule.w[k] * fabs(det) * manufactured_source(X, a.coeff_kind);
    }
    __syncthreads();
  }
  const double *qd = a.qd ? a.qd + e * qdata_estride(a.mode == 2 ? CEED_OP_DIFFUSION : CEED_OP_MASS, 8, Q) : nullptr;
  for (int n = threadIdx.x; n < nd; n += blockDim.x) {
    const int ia = n % P, ib = (n / P) % P, ic = n / (P * P);
    double val = 0.0;
    if (P == Q) {
      // collocated: B = I, so phi_n is nonzero at its own node only and its gradient lives on the
      // three lines of points through that node
      const int q0 = (ic * Q + ib) * Q + ia;
      if (a.mode == 0) {
        val = fq[q0];
      } else if (a.mode == 1) {
        val = qd[q0];
      } else {
        const double *D = a.tab.D;
        for (int m = 0; m < Q; ++m) {
          val += qd[(ic * Q + ib) * Q + m] * D[m * Q + ia] * D[m * Q + ia];
          val += qd[3 * nq + (ic * Q + m) * Q + ia] * D[m * Q + ib] * D[m * Q + ib];
          val += qd[5 * nq + (m * Q + ib) * Q + ia] * D[m * Q + ic] * D[m * Q + ic];
        }
        const double da = D[ia * Q + ia], db = D[ib * Q + ib], dc = D[ic * Q + ic];
        val += 2.0 * (qd[nq + q0] * da * db + qd[2 * nq + q0] * da * dc + qd[4 * nq + q0] * db * dc);
      }
    } else
    for (int k = 0; k < Q; ++k) {
      const double Bk = a.tab.B[k * P + ic], Gk = G1[k * P + ic];
      for (int j = 0; j < Q; ++j) {
        const double Bj = a.tab.B[j * P + ib], Gj = G1[j * P + ib];
        for (int i = 0; i < Q; ++i) {
          const double Bi = a.tab.B[i * P + ia], Gi = G1[i * P + ia];
          const int q = (k * Q + j) * Q + i;
          if (a.mode == 0) {
            val += Bi * Bj * Bk * fq[q];
          } else if (a.mode == 1) {
            const double ph = Bi * Bj * Bk;
            val += qd[q] * ph * ph;
          } else {
            const double gr = Gi * Bj * Bk, gs = Bi * Gj * Bk, gt = Bi * Bj * Gk;
            if (gr == 0.0 && gs == 0.0 && gt == 0.0) continue;
            val += qd[q] * gr * gr + qd[3 * nq + q] * gs * gs + qd[5 * nq + q] * gt * gt +
                   2.0 * (qd[nq + q] * gr * gs + qd[2 * nq + q] * gr * gt + qd[4 * nq + q] * gs * gt);
          }
        }
      }
    }
    const uint32_t v = a.emap[e * nd + n];
    const int64_t dof = v & DOF_MASK;
    for (int c = 0; c < a.ncomp; ++c) {
      double *o = a.out + dof * a.ncomp + c;
      if (a.masked && (v & FLAG_DIR)) {
        if (v & FLAG_FIRST) *o = (a.mode == 0) ? 0.0 : 1.0;
      } else if (v & FLAG_FIRST) {
        *o = val;
      } else {
        *o += val;
      }
    }
  }
}

static int run_elemvec(ceed_mesh_t m, ElemVecArgs a, cudaStream_t s) {
  a.emap = m->d_emap;
  a.vert = m->d_vertices;
  a.P = m->P;
  a.Q = m->Q;
  a.rule = m->rule;
  a.tab = m->tab64;
  const bool iso = a.mode == 0 && m->d_coords;
  a.coords = iso ? m->d_coords : nullptr;
  if (iso) a.iso = make_iso_tab(m);
  const size_t shm = ((size_t)nq_of(m) + MAX_Q * MAX_P + (iso ? iso_smem_doubles(m->P, m->Q) : 0)) * sizeof(double);
  if (int st = ensure_dynamic_smem((const void *)elemvec_kernel, shm)) return st;
  const int threads = iso ? ISO_THREADS : 128;
  for (int c = 0; c < m->n_colors; ++c) {
    a.e_begin = m->color_start[c];
    a.e_count = m->color_start[c + 1] - a.e_begin;
    if (a.e_count == 0) continue;
    elemvec_kernel<<<(unsigned)a.e_count, threads, shm, s>>>(a);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

}  // namespace ceedgb

using namespace ceedgb;

static int build_qdata_impl(ceed_mesh_t m, int op, int coeff_kind, const double *coeff, int prec, void *qdata,
                            cudaStream_t s) {
  if (int st = check_mesh(m)) return st;
  if (!qdata) return fail(CEED_ERR_INVALID, "null qdata");
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  double cconst = 1.0;
  if (coeff_kind == CEED_COEFF_CONST) {
    if (!coeff) return fail(CEED_ERR_INVALID, "CONST coefficient needs a host value");
    cconst = coeff[0];
  } else if (coeff_kind == CEED_COEFF_PER_QPT) {
    if (!coeff) return fail(CEED_ERR_INVALID, "PER_QPT coefficient needs a device array");
  } else if (coeff_kind != CEED_COEFF_ONE && coeff_kind != CEED_COEFF_SINE) {
    return fail(CEED_ERR_INVALID, "unknown coefficient kind");
  }
  CEED_CUDA_CHECK(cudaMemsetAsync(m->d_err, 0, sizeof(int), s));
  const int threads = 256;
  const int64_t total = m->E * nq_of(m);
  const unsigned blocks = (unsigned)std::min<int64_t>((total + threads - 1) / threads, 152 * 64);
  const QdataCoeff qc{op, coeff_kind, cconst, coeff, m->d_perm};
  if (prec == CEED_F32_GEO) {
    if (op != CEED_OP_DIFFUSION) return fail(CEED_ERR_UNSUPPORTED, "F32_GEO quadrature data is for diffusion");
    if (m->d_coords) return fail(CEED_ERR_UNSUPPORTED, "F32_GEO rebuilds the trilinear map; this mesh is curved");
    geo_qdata_kernel<<<blocks, threads, 0, s>>>(m->E, m->Q, m->d_vertices, m->d_perm, coeff_kind, cconst, coeff, m->rule,
                                                (float *)qdata, qdata_estride(OP_DIFF_GEO, 4, m->Q), m->d_err);
  } else {
    const IsoTab itab = m->d_coords ? make_iso_tab(m) : IsoTab{};
    const size_t ishm = (size_t)iso_smem_doubles(m->P, m->Q) * sizeof(double);
    const unsigned iblocks = (unsigned)std::min<int64_t>(m->E, 152 * 8);
#define CEEDGB_Q(TQ)                                                                                           \
  if (m->d_coords)                                                                                             \
    iso_qdata_kernel<TQ><<<iblocks, ISO_THREADS, ishm, s>>>(m->E, m->P, m->Q, m->d_emap, m->d_coords, itab, qc,   \
                                                           m->rule, (TQ *)qdata,                               \
                                                           qdata_estride(op, sizeof(TQ), m->Q), m->d_err);     \
  else                                                                                                         \
    qdata_kernel<TQ><<<blocks, threads, 0, s>>>(m->E, m->Q, m->d_vertices, qc, m->rule, (TQ *)qdata,             \
                                                qdata_estride(op, sizeof(TQ), m->Q), m->d_err)
  switch (prec) {
    case CEED_F64: CEEDGB_Q(double); break;
    case CEED_F32: CEEDGB_Q(float); break;
    case CEED_BF16: CEEDGB_Q(__nv_bfloat16); break;
    case CEED_F16: CEEDGB_Q(__half); break;
    case CEED_F64_DF: CEEDGB_Q(DF); break;
    default: return fail(CEED_ERR_INVALID, "unknown precision");
  }
#undef CEEDGB_Q
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  int err = 0;
  CEED_CUDA_CHECK(cudaMemcpyAsync(&err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  if (err) return fail(CEED_ERR_BAD_GEOMETRY, "det J <= 0 at some quadrature point");
  return CEED_OK;
}

extern "C" int ceed_build_qdata(ceed_mesh_t m, int op, int coeff_kind, const double *coeff, int prec, void *qdata,
                                void *stream) {
  return build_qdata_impl(m, op, coeff_kind, coeff, prec, qdata, (cudaStream_t)stream);
}

extern "C" int ceed_build_geometry(ceed_mesh_t m, void *geo, void *stream) {
  return build_qdata_impl(m, CEED_OP_DIFFUSION, CEED_COEFF_ONE, nullptr, CEED_F64, geo, (cudaStream_t)stream);
}

extern "C" int ceed_mesh_node_coords(ceed_mesh_t m, double *coords, void *stream) {
  if (int st = check_mesh(m)) return st;
  if (!coords) return fail(CEED_ERR_INVALID, "null coords");
  const cudaStream_t s = (cudaStream_t)stream;
  if (m->d_coords) {
    CEED_CUDA_CHECK(cudaMemcpyAsync(coords, m->d_coords, (size_t)m->n_ldof * 3 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
    return CEED_OK;
  }
  NodeCoordArgs a{};
  a.emap = m->d_emap;
  a.vert = m->d_vertices;
  a.coords = coords;
  a.E = m->E;
  a.P = m->P;
  for (int i = 0; i < m->P; ++i) a.x[i] = m->gll_x[i];
  const int64_t total = m->E * (int64_t)m->P * m->P * m->P;
  node_coords_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 64), 256, 0, s>>>(a);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

extern "C" int ceed_manufactured_rhs(ceed_mesh_t m, int coeff_kind, double *b, unsigned flags, void *stream) {
  if (int st = check_mesh(m)) return st;
  if (!b) return fail(CEED_ERR_INVALID, "null b");
  if (m->ncomp != 1) return fail(CEED_ERR_UNSUPPORTED, "manufactured RHS needs ncomp = 1");
  if (coeff_kind != CEED_COEFF_ONE && coeff_kind != CEED_COEFF_SINE)
    return fail(CEED_ERR_INVALID, "manufactured RHS supports ONE or SINE coefficients");
  ElemVecArgs a{};
  a.out = b;
  a.ncomp = 1;
  a.masked = (flags & CEED_APPLY_DIRICHLET) ? 1 : 0;
  if (a.masked && !m->has_dirichlet) return fail(CEED_ERR_INVALID, "mesh has no Dirichlet mask");
  a.mode = 0;
  a.coeff_kind = coeff_kind;
  return run_elemvec(m, a, (cudaStream_t)stream);
}

extern "C" int ceed_jacobi_diagonal(ceed_mesh_t m, int op, const void *qdata, int prec, double *diag, unsigned flags,
                                    void *stream) {
  if (int st = check_mesh(m)) return st;
  if (!qdata || !diag) return fail(CEED_ERR_INVALID, "null qdata or diag");
  if (prec != CEED_F64) return fail(CEED_ERR_UNSUPPORTED, "the Jacobi diagonal is built from FP64 quadrature data");
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  ElemVecArgs a{};
  a.qd = (const double *)qdata;
  a.out = diag;
  a.ncomp = m->ncomp;
  a.masked = (flags & CEED_APPLY_DIRICHLET) ? 1 : 0;
  if (a.masked && !m->has_dirichlet) return fail(CEED_ERR_INVALID, "mesh has no Dirichlet mask");
  a.mode = op == CEED_OP_MASS ? 1 : 2;
  return run_elemvec(m, a, (cudaStream_t)stream);
}
