// Non-tensor (simplex) elements: the basis-agnostic dense element operator of the paper's
// Section 3 (libCEED non-tensor bases; MAGMA backend).  The caller supplies the interpolation and
// gradient matrices of the basis at the quadrature points and the weights; the operator applies
// them element by element, y^e = B^T D B u^e (mass) or G^T D G u^e (diffusion), with the same
// pointwise D as the tensor-product path.  Two algorithms:
//   FUSED  one kernel per application: gather, forward contraction with the basis matrix,
//          pointwise D, transposed contraction, all in shared memory/registers, E-vector out;
//   GEMM   the paper's MAGMA formulation: the element inputs of all elements form one matrix, so
//          each basis action is one standard GEMM (cuBLAS; optionally split into a strided batch
//          of eta-element blocks), with the pointwise D in between.
// Both end with a deterministic transposed restriction: every L-vector node sums its element
// entries in a fixed order (no atomics, no colouring).
//
// Device layouts (element index fastest everywhere, so lanes of a warp read consecutive words):
//   restriction  uint32 [P][E]   node | FLAG_DIR
//   qdata        [ncomp][Q][E]   ncomp = 1 (mass) or 6 (diffusion: rr, rs, rt, ss, st, tt)
//   E-vectors    [P][E], [D*Q][E]
//   basis        [D][Q][P]       D = 1 (interp) or 3 (grad)
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "geometry.cuh"
#include "nontensor.h"

namespace ceedgb {

// ---------------------------------------------------------------------------------------------
// Host: the degree-p tetrahedron (helper for callers; the operator itself is basis-agnostic).

// Jacobi polynomial P_n^{(a,0)}(x) and its derivative, three-term recurrence (Szego, Orthogonal
// Polynomials, 4.5.1) and the derivative identity
// (2n+a)(1-x^2) P_n' = n (a - (2n+a) x) P_n + 2 n (n+a) P_{n-1}   (interior x).
static void jacobi_eval(int n, int a, double x, double *pn, double *dpn) {
  double p0 = 1.0, p1 = 0.5 * ((a + 2) * x + a);
  if (n == 0) {
    *pn = 1.0;
    *dpn = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double a1 = 2.0 * k * (k + a) * (2.0 * k + a - 2);
    const double a2 = (2.0 * k + a - 1) * a * a;
    const double a3 = (2.0 * k + a - 2) * (2.0 * k + a - 1) * (2.0 * k + a);
    const double a4 = 2.0 * (k + a - 1) * (k - 1) * (2.0 * k + a);
    const double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *dpn = (n * (a - (2.0 * n + a) * x) * p1 + 2.0 * n * (n + a) * p0) / ((2.0 * n + a) * (1.0 - x * x));
}

// n-point Gauss rule on [0, 1] for the weight (1 - u)^a: Newton with deflation on the roots of
// P_n^{(a,0)} in x = 2u - 1, weights 1 / ((1 - x^2) P_n'(x)^2) (the [-1, 1] Gauss-Jacobi weights
// 2^{a+1} / ((1 - x^2) P_n'^2) divided by the Jacobian 2^{a+1} of the map).
static void gauss_jacobi01(int n, int a, double *u, double *w) {
  const double pi = 3.14159265358979323846;
  std::vector<double> x(n);
  for (int k = 0; k < n; ++k) {
    double t = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
    if (k > 0 && t <= x[k - 1]) t = 0.5 * (x[k - 1] + 1.0);
    for (int it = 0; it < 200; ++it) {
      double p, dp;
      jacobi_eval(n, a, t, &p, &dp);
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (t - x[j]);
      const double dt = p / (dp - p * s);
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[k] = t;
  }
  std::sort(x.begin(), x.end());
  for (int k = 0; k < n; ++k) {
    double p, dp;
    jacobi_eval(n, a, x[k], &p, &dp);
    u[k] = 0.5 * (1.0 + x[k]);
    w[k] = 1.0 / ((1.0 - x[k] * x[k]) * dp * dp);
  }
}

// Silvester's factor R_m(t) = prod_{s<m} (p t - s) / (s + 1) and its derivative.
static void silvester(int m, int p, double t, double *R, double *dR) {
  double r = 1.0, d = 0.0;
  for (int s = 0; s < m; ++s) {
    const double f = (p * t - s) / (s + 1.0);
    d = d * f + r * p / (s + 1.0);   // product rule, accumulated factor by factor
    r *= f;
  }
  *R = r;
  *dR = d;
}

}  // namespace ceedgb

using namespace ceedgb;

extern "C" int ceed_simplex_sizes(int p, int q, int32_t *P, int32_t *Q) {
  if (p < 1 || p > 7) return fail(CEED_ERR_INVALID, "simplex basis: p must be in 1..7");
  if (q < 1 || q > 10) return fail(CEED_ERR_INVALID, "simplex basis: q must be in 1..10");
  if (P) *P = (p + 1) * (p + 2) * (p + 3) / 6;
  if (Q) *Q = q * q * q;
  return CEED_OK;
}

extern "C" int ceed_simplex_basis(int p, int q, double *interp, double *grad, double *qweight, double *qref) {
  int32_t P, Q;
  int st = ceed_simplex_sizes(p, q, &P, &Q);
  if (st != CEED_OK) return st;
  // conical product rule: xi = (u, (1-u) v, (1-u)(1-v) w), weights of (1-u)^2, (1-v), 1
  double u[10], wu[10], v[10], wv[10], t[10], wt[10];
  gauss_jacobi01(q, 2, u, wu);
  gauss_jacobi01(q, 1, v, wv);
  gauss_jacobi01(q, 0, t, wt);
  std::vector<double> xi(3 * (size_t)Q);
  for (int c = 0; c < q; ++c)
    for (int b = 0; b < q; ++b)
      for (int a = 0; a < q; ++a) {
        const int k = a + q * (b + q * c);
        xi[3 * k + 0] = u[a];
        xi[3 * k + 1] = (1.0 - u[a]) * v[b];
        xi[3 * k + 2] = (1.0 - u[a]) * (1.0 - v[b]) * t[c];
        if (qweight) qweight[k] = wu[a] * wv[b] * wt[c];
      }
  if (qref) std::memcpy(qref, xi.data(), xi.size() * sizeof(double));
  // nodes (i, j, k), k slowest, i fastest; alpha = (p - i - j - k, i, j, k) on the barycentric
  // coordinates (1 - xi_1 - xi_2 - xi_3, xi_1, xi_2, xi_3)
  int n = 0;
  for (int kk = 0; kk <= p; ++kk)
    for (int jj = 0; jj <= p - kk; ++jj)
      for (int ii = 0; ii <= p - jj - kk; ++ii, ++n) {
        const int al[4] = {p - ii - jj - kk, ii, jj, kk};
        for (int k = 0; k < Q; ++k) {
          const double lam[4] = {1.0 - xi[3 * k] - xi[3 * k + 1] - xi[3 * k + 2], xi[3 * k], xi[3 * k + 1],
                                 xi[3 * k + 2]};
          double R[4], dR[4];
          for (int m = 0; m < 4; ++m) silvester(al[m], p, lam[m], &R[m], &dR[m]);
          double dl[4];
          for (int m = 0; m < 4; ++m) {
            dl[m] = dR[m];
            for (int o = 0; o < 4; ++o)
              if (o != m) dl[m] *= R[o];
          }
          if (interp) interp[(size_t)k * P + n] = R[0] * R[1] * R[2] * R[3];
          if (grad)
            for (int d = 0; d < 3; ++d) grad[((size_t)d * Q + k) * P + n] = dl[d + 1] - dl[0];
        }
      }
  return CEED_OK;
}

namespace ceedgb {

// ---------------------------------------------------------------------------------------------
// Device kernels.

template <typename T>
__device__ __forceinline__ T nt_cvt(double v);
template <>
__device__ __forceinline__ double nt_cvt<double>(double v) { return v; }
template <>
__device__ __forceinline__ float nt_cvt<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ DF nt_cvt<DF>(double v) { return df_from_double(v); }

__device__ __forceinline__ double nt_to_double(double v) { return v; }
__device__ __forceinline__ double nt_to_double(float v) { return (double)v; }
__device__ __forceinline__ double nt_to_double(DF v) { return (double)v.hi + (double)v.lo; }

// Quadrature data of the affine simplex map x = v0 + J xi (J columns v1-v0, v2-v0, v3-v0): mass
// w |det J| rho, diffusion w k adj(J) adj(J)^T / det J.  One thread per (point, element).
template <typename T>
__global__ void nt_qdata_kernel(int64_t E, int64_t Es, int Q, int op, const double *__restrict__ vert,
                                const double *__restrict__ qw, const double *__restrict__ qref, int coeff_kind,
                                double cconst, const double *__restrict__ coeff, T *__restrict__ out, int *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Es * Q) return;
  const int64_t e = i % Es;
  const int q = (int)(i / Es);
  const int64_t cs = (int64_t)Q * Es;
  T *o = out + (int64_t)q * Es + e;
  if (e >= E) {   // padding of the last tile: zeros
    for (int k = 0; k < (op == CEED_OP_MASS ? 1 : 6); ++k) o[k * cs] = T(0);
    return;
  }
  const double *V = vert + e * 12;
  double J[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) J[a][b] = V[3 * (b + 1) + a] - V[a];
  double A[3][3];
  const double det = adjugate(J, A);
  if (!(det > 0.0)) *err = CEED_ERR_BAD_GEOMETRY;
  double k = 1.0;
  if (coeff_kind == CEED_COEFF_CONST) {
    k = cconst;
  } else if (coeff_kind == CEED_COEFF_SINE) {
    double X[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      X[a] = V[a] + J[a][0] * qref[3 * q] + J[a][1] * qref[3 * q + 1] + J[a][2] * qref[3 * q + 2];
    k = sine_coefficient(X);
  } else if (coeff_kind == CEED_COEFF_PER_QPT) {
    k = coeff[e * Q + q];
  }
  const double w = qw[q];
  if (op == CEED_OP_MASS) {
    o[0] = nt_cvt<T>(w * fabs(det) * k);
  } else {
    const double f = w * k / det;
    o[0 * cs] = nt_cvt<T>(f * (A[0][0] * A[0][0] + A[0][1] * A[0][1] + A[0][2] * A[0][2]));
    o[1 * cs] = nt_cvt<T>(f * (A[0][0] * A[1][0] + A[0][1] * A[1][1] + A[0][2] * A[1][2]));
    o[2 * cs] = nt_cvt<T>(f * (A[0][0] * A[2][0] + A[0][1] * A[2][1] + A[0][2] * A[2][2]));
    o[3 * cs] = nt_cvt<T>(f * (A[1][0] * A[1][0] + A[1][1] * A[1][1] + A[1][2] * A[1][2]));
    o[4 * cs] = nt_cvt<T>(f * (A[1][0] * A[2][0] + A[1][1] * A[2][1] + A[1][2] * A[2][2]));
    o[5 * cs] = nt_cvt<T>(f * (A[2][0] * A[2][0] + A[2][1] * A[2][1] + A[2][2] * A[2][2]));
  }
}

// Pointwise quadrature operator on one point: mass v = qd u; diffusion v = G g (G symmetric 3x3
// from its six stored entries).
template <typename T, int D>
__device__ __forceinline__ void nt_pointwise(const T *__restrict__ qd, int64_t cs, T g[D]) {
  if (D == 1) {
    g[0] *= qd[0];
  } else {
    const T c0 = qd[0], c1 = qd[cs], c2 = qd[2 * cs], c3 = qd[3 * cs], c4 = qd[4 * cs], c5 = qd[5 * cs];
    const T g0 = g[0], g1 = g[1], g2 = g[2];
    g[0] = c0 * g0 + c1 * g1 + c2 * g2;
    g[1] = c1 * g0 + c3 * g1 + c4 * g2;
    g[2] = c2 * g0 + c4 * g1 + c5 * g2;
  }
}

// Fused element operator: NT_NE elements per block (element = lane), 8 warps.  The block gathers
// its elements' inputs into shared memory, then walks the quadrature points in chunks of NT_QC:
// stage the chunk's rows of the basis matrix, forward contraction S = B u (rows spread over the
// warps, the basis entry a broadcast, the input a conflict-free row), pointwise D on S with the
// quadrature data read coalesced (element fastest), and the transposed contraction accumulated
// in registers (node rows spread over the warps).  Output: the element vectors, [P][E].
template <typename T, int D>
__global__ void __launch_bounds__(NT_NE * NT_WARPS)
    nt_fused_kernel(int64_t E, int64_t Es, int P, int Q, const uint32_t *__restrict__ rmap, const double *__restrict__ x,
                    const T *__restrict__ tab, const T *__restrict__ qd, T *__restrict__ Ye, int masked) {
  extern __shared__ __align__(16) unsigned char nt_smem[];
  T *Us = reinterpret_cast<T *>(nt_smem);   // [P][NT_NE]
  T *Gc = Us + P * NT_NE;                    // [D][NT_QC][P]
  T *Sv = Gc + D * NT_QC * P;                // [D NT_QC][NT_NE + 1]
  constexpr int LD = NT_NE + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * NT_NE + lane;
  const bool valid = e < E;
  for (int n = warp; n < P; n += NT_WARPS) {
    T v = T(0);
    if (valid) {
      const uint32_t m = rmap[(int64_t)n * E + e];
      if (!(masked && (m & FLAG_DIR))) v = nt_cvt<T>(x[m & DOF_MASK]);
    }
    Us[n * NT_NE + lane] = v;
  }
  T yr[NT_YR];
#pragma unroll
  for (int j = 0; j < NT_YR; ++j) yr[j] = T(0);
  const int64_t cs = (int64_t)Q * Es;
  for (int q0 = 0; q0 < Q; q0 += NT_QC) {
    const int qc = min(NT_QC, Q - q0);
    __syncthreads();
    for (int i = threadIdx.x; i < D * qc * P; i += NT_NE * NT_WARPS) {
      const int d = i / (qc * P), r = i - d * qc * P;
      Gc[d * NT_QC * P + r] = tab[((int64_t)d * Q + q0) * P + r];
    }
    __syncthreads();
    for (int r = warp; r < D * NT_QC; r += NT_WARPS) {
      if (r % NT_QC >= qc) continue;
      const T *g = Gc + r * P;
      T a0 = T(0), a1 = T(0);
      int n = 0;
      for (; n + 1 < P; n += 2) {
        a0 = fma(g[n], Us[n * NT_NE + lane], a0);
        a1 = fma(g[n + 1], Us[(n + 1) * NT_NE + lane], a1);
      }
      if (n < P) a0 = fma(g[n], Us[n * NT_NE + lane], a0);
      Sv[r * LD + lane] = a0 + a1;
    }
    __syncthreads();
    for (int q = warp; q < qc; q += NT_WARPS) {
      T g[D];
#pragma unroll
      for (int d = 0; d < D; ++d) g[d] = Sv[(d * NT_QC + q) * LD + lane];
      if (valid) {
        nt_pointwise<T, D>(qd + (int64_t)(q0 + q) * Es + e, cs, g);
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) g[d] = T(0);
      }
#pragma unroll
      for (int d = 0; d < D; ++d) Sv[(d * NT_QC + q) * LD + lane] = g[d];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NT_YR; ++j) {
      const int n = warp + NT_WARPS * j;
      if (n < P) {
        T acc = yr[j];
        for (int d = 0; d < D; ++d) {
          const T *g = Gc + d * NT_QC * P + n;
          const T *s = Sv + d * NT_QC * LD + lane;
          for (int q = 0; q < qc; ++q) acc = fma(g[q * P], s[q * LD], acc);
        }
        yr[j] = acc;
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int j = 0; j < NT_YR; ++j) {
      const int n = warp + NT_WARPS * j;
      if (n < P) Ye[(int64_t)n * E + e] = yr[j];
    }
  }
}

// GEMM path, step 1: element inputs U [P][E] from the L-vector.
template <typename T>
__global__ void nt_gather_kernel(int64_t total, const uint32_t *__restrict__ rmap, const double *__restrict__ x,
                                 T *__restrict__ U, int masked) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const uint32_t m = rmap[i];
  U[i] = (masked && (m & FLAG_DIR)) ? T(0) : nt_cvt<T>(x[m & DOF_MASK]);
}

// GEMM path, step 3: pointwise D in place on S [D][Q][E]; grid x over elements, y over points.
template <typename T, int D>
__global__ void nt_pointwise_kernel(int64_t E, int64_t Es, int Q, const T *__restrict__ qd, T *__restrict__ S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (e >= E) return;
  const int64_t cs = (int64_t)Q * E, i = (int64_t)q * E + e;
  T g[D];
#pragma unroll
  for (int d = 0; d < D; ++d) g[d] = S[d * cs + i];
  nt_pointwise<T, D>(qd + (int64_t)q * Es + e, (int64_t)Q * Es, g);
#pragma unroll
  for (int d = 0; d < D; ++d) S[d * cs + i] = g[d];
}

// Transposed restriction: y_i = sum of node i's element entries in ascending position order
// (deterministic); with masking, y_i = x_i on Dirichlet nodes.
template <typename T>
__global__ void nt_assemble_kernel(int64_t n, const int64_t *__restrict__ off, const uint32_t *__restrict__ pos,
                                   const T *__restrict__ Ye, const uint8_t *__restrict__ dir,
                                   const double *__restrict__ x, double *__restrict__ y, int masked) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (masked && dir[i]) {
    y[i] = x[i];
    return;
  }
  double acc = 0.0;
  for (int64_t k = off[i]; k < off[i + 1]; ++k) acc += nt_to_double(Ye[pos[k]]);
  y[i] = acc;
}

// The fused kernel with FP64 accuracy on the FP32 pipe: values and tables as double-float pairs, every
// contraction and the pointwise products as compensated dot products (Dot2, df.cuh), the same data
// flow as nt_fused_kernel.  The forward sums run as two Dot2 chains (even and odd basis functions)
// joined by a double-float addition; the transposed sums accumulate in one Dot2 chain per node.
template <int D>
__global__ void __launch_bounds__(NT_NE * NT_WARPS)
    nt_fused_df_kernel(int64_t E, int64_t Es, int P, int Q, const uint32_t *__restrict__ rmap,
                       const double *__restrict__ x, const DF *__restrict__ tab, const DF *__restrict__ qd,
                       DF *__restrict__ Ye, int masked) {
  extern __shared__ __align__(16) unsigned char nt_smem[];
  DF *Us = reinterpret_cast<DF *>(nt_smem);  // [P][NT_NE]
  DF *Gc = Us + P * NT_NE;                     // [D][NT_QC][P]
  DF *Sv = Gc + D * NT_QC * P;                 // [D NT_QC][NT_NE + 1]
  constexpr int LD = NT_NE + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * NT_NE + lane;
  const bool valid = e < E;
  for (int n = warp; n < P; n += NT_WARPS) {
    DF v(0.f, 0.f);
    if (valid) {
      const uint32_t m = rmap[(int64_t)n * E + e];
      if (!(masked && (m & FLAG_DIR))) v = nt_cvt<DF>(x[m & DOF_MASK]);
    }
    Us[n * NT_NE + lane] = v;
  }
  DFAcc yr[NT_YR];
#pragma unroll
  for (int j = 0; j < NT_YR; ++j) yr[j] = DFAcc{0.f, 0.f};
  const int64_t cs = (int64_t)Q * Es;
  for (int q0 = 0; q0 < Q; q0 += NT_QC) {
    const int qc = min(NT_QC, Q - q0);
    __syncthreads();
    for (int i = threadIdx.x; i < D * qc * P; i += NT_NE * NT_WARPS) {
      const int d = i / (qc * P), r = i - d * qc * P;
      Gc[d * NT_QC * P + r] = tab[((int64_t)d * Q + q0) * P + r];
    }
    __syncthreads();
    for (int r = warp; r < D * NT_QC; r += NT_WARPS) {
      if (r % NT_QC >= qc) continue;
      const DF *g = Gc + r * P;
      DFAcc a0 = acc_first(g[0], Us[lane]);
      DFAcc a1{0.f, 0.f};
      int n = 1;
      if (P > 1) {
        a1 = acc_first(g[1], Us[NT_NE + lane]);
        for (n = 2; n + 1 < P; n += 2) {
          acc_mac(a0, g[n], Us[n * NT_NE + lane]);
          acc_mac(a1, g[n + 1], Us[(n + 1) * NT_NE + lane]);
        }
      }
      if (n < P) acc_mac(a0, g[n], Us[n * NT_NE + lane]);
      Sv[r * LD + lane] = df_add(acc_get(a0), acc_get(a1));
    }
    __syncthreads();
    for (int q = warp; q < qc; q += NT_WARPS) {
      DF g[D];
#pragma unroll
      for (int d = 0; d < D; ++d) g[d] = Sv[(d * NT_QC + q) * LD + lane];
      if (valid) {
        const DF *c = qd + (int64_t)(q0 + q) * Es + e;
        if (D == 1) {
          g[0] = acc_get(acc_first(c[0], g[0]));
        } else {
          const DF c0 = c[0], c1 = c[cs], c2 = c[2 * cs], c3 = c[3 * cs], c4 = c[4 * cs], c5 = c[5 * cs];
          const DF g0 = g[0], g1 = g[1], g2 = g[2];
          DFAcc A = acc_first(c0, g0), B = acc_first(c1, g0), C = acc_first(c2, g0);
          acc_mac(A, c1, g1);
          acc_mac(B, c3, g1);
          acc_mac(C, c4, g1);
          acc_mac(A, c2, g2);
          acc_mac(B, c4, g2);
          acc_mac(C, c5, g2);
          g[0] = acc_get(A);
          g[1] = acc_get(B);
          g[2] = acc_get(C);
        }
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) g[d] = DF(0.f, 0.f);
      }
#pragma unroll
      for (int d = 0; d < D; ++d) Sv[(d * NT_QC + q) * LD + lane] = g[d];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NT_YR; ++j) {
      const int n = warp + NT_WARPS * j;
      if (n < P) {
        DFAcc acc = yr[j];
        for (int d = 0; d < D; ++d) {
          const DF *g = Gc + d * NT_QC * P + n;
          const DF *sv = Sv + d * NT_QC * LD + lane;
          for (int q = 0; q < qc; ++q) acc_mac(acc, g[q * P], sv[q * LD]);
        }
        yr[j] = acc;
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int j = 0; j < NT_YR; ++j) {
      const int n = warp + NT_WARPS * j;
      if (n < P) Ye[(int64_t)n * E + e] = acc_get(yr[j]);
    }
  }
}

static size_t nt_fused_smem(int P, int D, size_t tsize) {
  return tsize * ((size_t)P * NT_NE + (size_t)D * NT_QC * P + (size_t)D * NT_QC * (NT_NE + 1));
}

template <typename T, int D>
static int launch_fused(ceed_nt_t h, const T *tab, const T *qd, const double *x, T *Ye, int masked, cudaStream_t s) {
  const size_t sm = nt_fused_smem(h->P, D, sizeof(T));
  if (int st = ensure_dynamic_smem((const void *)nt_fused_kernel<T, D>, 227 * 1024)) return st;
  const unsigned grid = (unsigned)((h->E + NT_NE - 1) / NT_NE);
  nt_fused_kernel<T, D><<<grid, NT_NE * NT_WARPS, sm, s>>>(h->E, h->Es, h->P, h->Q, h->d_rmap, x, tab, qd, Ye, masked);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

static int blas_fail(cublasStatus_t st, const char *where) {
  return fail(st == CUBLAS_STATUS_ALLOC_FAILED ? CEED_ERR_OOM : CEED_ERR_CUDA,
              std::string(where) + ": cuBLAS status " + std::to_string((int)st));
}

// C [rows x n] (column-major, leading dimension E) = A [rows x k] (ld E) * op(B), B the basis matrix
// as a column-major [P x D Q] array (ld P).  eta > 0 splits the rows into a strided batch.
template <typename T>
static int nt_gemm(ceed_nt_t h, bool transB, int m_n, int m_k, const T *A, const T *B, T *C, int64_t eta, int mode) {
  const cudaDataType_t dt = sizeof(T) == 8 ? CUDA_R_64F : CUDA_R_32F;
  cublasComputeType_t ct;
  if (sizeof(T) == 8) ct = mode == 1 ? CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT : CUBLAS_COMPUTE_64F;
  else ct = mode == 1 ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : mode == 2 ? CUBLAS_COMPUTE_32F_FAST_TF32 : CUBLAS_COMPUTE_32F;
  // the handle's math mode admits the emulated algorithms only when they are asked for
  cublasMath_t mm = CUBLAS_DEFAULT_MATH;
  if (mode == 1) mm = sizeof(T) == 8 ? CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH : CUBLAS_FP32_EMULATED_BF16X9_MATH;
  else if (mode == 2) mm = CUBLAS_TF32_TENSOR_OP_MATH;
  cublasStatus_t ms = cublasSetMathMode(h->blas, mm);
  if (ms != CUBLAS_STATUS_SUCCESS) return blas_fail(ms, "cublasSetMathMode");
  const T one = T(1), zero = T(0);
  const int64_t E = h->E;
  const cublasOperation_t ob = transB ? CUBLAS_OP_T : CUBLAS_OP_N;
  const int ldb = h->P;
  cublasStatus_t st;
  if (eta <= 0 || eta >= E) {
    st = cublasGemmEx(h->blas, CUBLAS_OP_N, ob, (int)E, m_n, m_k, &one, A, dt, (int)E, B, dt, ldb, &zero, C, dt, (int)E,
                      ct, CUBLAS_GEMM_DEFAULT);
    if (st != CUBLAS_STATUS_SUCCESS) return blas_fail(st, "cublasGemmEx");
    return CEED_OK;
  }
  const int64_t nb = E / eta, rem = E - nb * eta;
  st = cublasGemmStridedBatchedEx(h->blas, CUBLAS_OP_N, ob, (int)eta, m_n, m_k, &one, A, dt, (int)E, eta, B, dt, ldb, 0,
                                  &zero, C, dt, (int)E, eta, (int)nb, ct, CUBLAS_GEMM_DEFAULT);
  if (st != CUBLAS_STATUS_SUCCESS) return blas_fail(st, "cublasGemmStridedBatchedEx");
  if (rem > 0) {
    st = cublasGemmEx(h->blas, CUBLAS_OP_N, ob, (int)rem, m_n, m_k, &one, A + nb * eta, dt, (int)E, B, dt, ldb, &zero,
                      C + nb * eta, dt, (int)E, ct, CUBLAS_GEMM_DEFAULT);
    if (st != CUBLAS_STATUS_SUCCESS) return blas_fail(st, "cublasGemmEx (remainder)");
  }
  return CEED_OK;
}

static int nt_ensure_gemm_workspace(ceed_nt_t h) {
  if (h->d_u) return CEED_OK;
  CEED_CUDA_CHECK(cudaMalloc(&h->d_u, (size_t)h->P * h->E * sizeof(double)));
  const cudaError_t e = cudaMalloc(&h->d_s, (size_t)3 * h->Q * h->E * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(h->d_u);
    h->d_u = nullptr;
    return cuda_fail(e, "cudaMalloc (GEMM workspace)");
  }
  return CEED_OK;
}

template <typename T, int D>
static int nt_apply_t(ceed_nt_t h, const NtChoice &c, const T *tab, const T *qd, const double *x, double *y, int masked,
                      cudaStream_t s) {
  T *Ye = reinterpret_cast<T *>(h->d_evec);
  int st;
  if (c.algo == CEED_NT_FUSED) {
    st = launch_fused<T, D>(h, tab, qd, x, Ye, masked, s);
  } else if (c.algo == CEED_NT_TC) {
    if (sizeof(T) != 4) return fail(CEED_ERR_UNSUPPORTED, "tensor-core algorithm: F32 only");
    st = nt_tc_apply(h, D == 1 ? CEED_OP_MASS : CEED_OP_DIFFUSION, reinterpret_cast<const float *>(qd), x,
                     reinterpret_cast<float *>(Ye), masked, s);
  } else {
    if ((st = nt_ensure_gemm_workspace(h)) != CEED_OK) return st;
    T *U = reinterpret_cast<T *>(h->d_u), *S = reinterpret_cast<T *>(h->d_s);
    const int64_t tot = (int64_t)h->P * h->E;
    nt_gather_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(tot, h->d_rmap, x, U, masked);
    CEED_CUDA_CHECK(cudaGetLastError());
    cublasStatus_t bs = cublasSetStream(h->blas, s);
    if (bs != CUBLAS_STATUS_SUCCESS) return blas_fail(bs, "cublasSetStream");
    if ((st = nt_gemm<T>(h, false, D * h->Q, h->P, U, tab, S, c.eta, c.gemm_mode)) != CEED_OK) return st;
    nt_pointwise_kernel<T, D><<<dim3((unsigned)((h->E + 255) / 256), (unsigned)h->Q), 256, 0, s>>>(h->E, h->Es, h->Q,
                                                                                               qd, S);
    CEED_CUDA_CHECK(cudaGetLastError());
    st = nt_gemm<T>(h, true, h->P, D * h->Q, S, tab, Ye, c.eta, c.gemm_mode);
  }
  if (st != CEED_OK) return st;
  nt_assemble_kernel<T><<<(unsigned)((h->n_ldof + 255) / 256), 256, 0, s>>>(h->n_ldof, h->d_off, h->d_pos, Ye,
                                                                             h->d_dir, x, y, masked);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

static int nt_apply(ceed_nt_t h, int op, const void *qdata, int prec, const double *x, double *y, unsigned flags,
                    const NtChoice &c, cudaStream_t s) {
  const int masked = (flags & CEED_APPLY_DIRICHLET) && h->has_dirichlet;
  const size_t tab_off = (size_t)(op == CEED_OP_MASS ? 0 : 1) * h->Q * h->P;
  if (prec == CEED_F64) {
    const double *tab = h->d_tab64 + tab_off;
    const double *qd = static_cast<const double *>(qdata);
    return op == CEED_OP_MASS ? nt_apply_t<double, 1>(h, c, tab, qd, x, y, masked, s)
                              : nt_apply_t<double, 3>(h, c, tab, qd, x, y, masked, s);
  }
  if (prec == CEED_F64_DF) {  // the fused double-float kernel (the only algorithm of this precision)
    const DF *tab = h->d_tabdf + tab_off;
    const DF *qd = static_cast<const DF *>(qdata);
    DF *Ye = reinterpret_cast<DF *>(h->d_evec);
    const int D = op == CEED_OP_MASS ? 1 : 3;
    const size_t sm = nt_fused_smem(h->P, D, sizeof(DF));
    const void *kfn = D == 1 ? (const void *)nt_fused_df_kernel<1> : (const void *)nt_fused_df_kernel<3>;
    if (int st = ensure_dynamic_smem(kfn, 227 * 1024)) return st;
    const unsigned grid = (unsigned)((h->E + NT_NE - 1) / NT_NE);
    if (D == 1)
      nt_fused_df_kernel<1><<<grid, NT_NE * NT_WARPS, sm, s>>>(h->E, h->Es, h->P, h->Q, h->d_rmap, x, tab, qd, Ye, masked);
    else
      nt_fused_df_kernel<3><<<grid, NT_NE * NT_WARPS, sm, s>>>(h->E, h->Es, h->P, h->Q, h->d_rmap, x, tab, qd, Ye, masked);
    CEED_CUDA_CHECK(cudaGetLastError());
    nt_assemble_kernel<DF><<<(unsigned)((h->n_ldof + 255) / 256), 256, 0, s>>>(h->n_ldof, h->d_off, h->d_pos, Ye,
                                                                                h->d_dir, x, y, masked);
    CEED_CUDA_CHECK(cudaGetLastError());
    return CEED_OK;
  }
  const float *tab = h->d_tab32 + tab_off;
  const float *qd = static_cast<const float *>(qdata);
  return op == CEED_OP_MASS ? nt_apply_t<float, 1>(h, c, tab, qd, x, y, masked, s)
                            : nt_apply_t<float, 3>(h, c, tab, qd, x, y, masked, s);
}

static int nt_check(ceed_nt_t h, int op, int prec) {
  if (!h) return fail(CEED_ERR_INVALID, "null non-tensor operator handle");
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "op must be MASS or DIFFUSION");
  if (prec != CEED_F64 && prec != CEED_F32 && prec != CEED_F64_DF)
    return fail(CEED_ERR_UNSUPPORTED, "non-tensor operator: prec F64, F32 or F64_DF");
  return CEED_OK;
}

// slot of a precision in the handle's algorithm choices
static int nt_slot(int prec) { return prec == CEED_F64 ? 0 : prec == CEED_F32 ? 1 : 2; }

}  // namespace ceedgb

namespace {
struct NtFree {
  void operator()(ceed_nt_s *h) const {
    if (!h) return;
    if (h->blas) cublasDestroy(h->blas);
    cudaFree(h->d_tab64);
    cudaFree(h->d_tab32);
    cudaFree(h->d_tabdf);
    cudaFree(h->d_qw);
    cudaFree(h->d_qref);
    cudaFree(h->d_rmap);
    cudaFree(h->d_off);
    cudaFree(h->d_pos);
    cudaFree(h->d_dir);
    cudaFree(h->d_vert);
    cudaFree(h->d_err);
    cudaFree(h->d_evec);
    cudaFree(h->d_u);
    cudaFree(h->d_s);
    cudaFree(h->d_tc_tab[0]);
    cudaFree(h->d_tc_tab[1]);
    delete h;
  }
};
}  // namespace

extern "C" int ceed_nt_setup(const ceed_nt_desc *desc, ceed_nt_t *out, void *stream) {
  if (!desc || !out) return fail(CEED_ERR_INVALID, "null descriptor or output");
  *out = nullptr;
  const int64_t E = desc->n_elem, nL = desc->n_ldof;
  const int P = desc->P, Q = desc->Q;
  if (E < 1 || nL < 1) return fail(CEED_ERR_INVALID, "n_elem and n_ldof must be >= 1");
  if (nL > (int64_t)DOF_MASK) return fail(CEED_ERR_INVALID, "n_ldof must be < 2^29");
  if (P < 1 || P > NT_MAXP) return fail(CEED_ERR_INVALID, "P must be in 1..128");
  if (Q < 1 || Q > NT_MAXQ) return fail(CEED_ERR_INVALID, "Q must be in 1..1024");
  if ((int64_t)P * E >= ((int64_t)1 << 32) || (int64_t)3 * Q * (E + 127) >= ((int64_t)1 << 31))
    return fail(CEED_ERR_INVALID, "mesh too large for 32-bit element-vector positions");
  if (!desc->interp || !desc->grad || !desc->qweight || !desc->qref)
    return fail(CEED_ERR_INVALID, "interp, grad, qweight and qref (host arrays) are required");
  if (!desc->elem_dofs || !desc->vertices) return fail(CEED_ERR_INVALID, "elem_dofs and vertices are required");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<ceed_nt_s, NtFree> h(new (std::nothrow) ceed_nt_s());
  if (!h) return fail(CEED_ERR_OOM, "host allocation");
  CEED_CUDA_CHECK(cudaGetDevice(&h->device));
  h->E = E;
  h->Es = (E + 127) / 128 * 128;
  h->n_ldof = nL;
  h->P = P;
  h->Q = Q;
  h->has_dirichlet = desc->dirichlet != nullptr;

  std::vector<int32_t> map;
  std::vector<uint8_t> dir;
  std::vector<uint32_t> rmap;
  std::vector<int64_t> off;
  std::vector<uint32_t> pos;
  std::vector<double> tab64;
  std::vector<float> tab32;
  try {
    map.resize((size_t)E * P);
    dir.assign(nL, 0);
    rmap.resize((size_t)E * P);
    off.assign(nL + 1, 0);
    pos.resize((size_t)E * P);
    tab64.resize((size_t)4 * Q * P);
    tab32.resize((size_t)4 * Q * P);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation for the mesh copy");
  }
  CEED_CUDA_CHECK(cudaMemcpyAsync(map.data(), desc->elem_dofs, (size_t)E * P * 4, cudaMemcpyDeviceToHost, s));
  if (desc->dirichlet) CEED_CUDA_CHECK(cudaMemcpyAsync(dir.data(), desc->dirichlet, nL, cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  for (int64_t v = 0; v < nL; ++v) dir[v] = dir[v] ? 1 : 0;

  // validate (in range, no node twice in an element, every node referenced) and count entries per node
  {
    std::vector<int64_t> stamp;
    try {
      stamp.assign(nL, -1);
    } catch (...) {
      return fail(CEED_ERR_OOM, "host allocation");
    }
    for (int64_t e = 0; e < E; ++e)
      for (int n = 0; n < P; ++n) {
        const int64_t v = map[e * P + n];
        if (v < 0 || v >= nL) return fail(CEED_ERR_INVALID, "elem_dofs entry out of range at element " + std::to_string(e));
        if (stamp[v] == e) return fail(CEED_ERR_INVALID, "node repeated inside element " + std::to_string(e));
        stamp[v] = e;
        off[v + 1]++;
      }
    for (int64_t v = 0; v < nL; ++v)
      if (stamp[v] < 0) return fail(CEED_ERR_INVALID, "node " + std::to_string(v) + " belongs to no element");
  }
  for (int64_t v = 0; v < nL; ++v) off[v + 1] += off[v];
  {
    // positions n E + e in ascending order per node (fill in increasing position order)
    std::vector<int64_t> fillp(off.begin(), off.end() - 1);
    for (int n = 0; n < P; ++n)
      for (int64_t e = 0; e < E; ++e) {
        const int64_t v = map[e * P + n];
        rmap[(size_t)n * E + e] = (uint32_t)v | (dir[v] ? FLAG_DIR : 0u);
        pos[fillp[v]++] = (uint32_t)((int64_t)n * E + e);
      }
  }
  // basis tables [4][Q][P]: interp, grad_1, grad_2, grad_3
  for (size_t i = 0; i < (size_t)Q * P; ++i) tab64[i] = desc->interp[i];
  for (size_t i = 0; i < (size_t)3 * Q * P; ++i) tab64[(size_t)Q * P + i] = desc->grad[i];
  for (size_t i = 0; i < tab64.size(); ++i) tab32[i] = (float)tab64[i];
  std::vector<DF> tabdf(tab64.size());
  for (size_t i = 0; i < tab64.size(); ++i) tabdf[i] = df_from_double(tab64[i]);

  CEED_CUDA_CHECK(cudaMalloc(&h->d_tab64, tab64.size() * 8));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_tab32, tab32.size() * 4));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_tabdf, tabdf.size() * sizeof(DF)));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_qw, (size_t)Q * 8));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_qref, (size_t)Q * 24));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_rmap, rmap.size() * 4));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_off, off.size() * 8));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_pos, pos.size() * 4));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_dir, (size_t)nL));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_vert, (size_t)E * 96));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_err, sizeof(int)));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_evec, (size_t)P * E * 8));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_tab64, tab64.data(), tab64.size() * 8, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_tab32, tab32.data(), tab32.size() * 4, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_tabdf, tabdf.data(), tabdf.size() * sizeof(DF), cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_qw, desc->qweight, (size_t)Q * 8, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_qref, desc->qref, (size_t)Q * 24, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_rmap, rmap.data(), rmap.size() * 4, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_pos, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_dir, dir.data(), (size_t)nL, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(h->d_vert, desc->vertices, (size_t)E * 96, cudaMemcpyDeviceToDevice, s));
  CEED_CUDA_CHECK(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  cublasStatus_t bs = cublasCreate(&h->blas);
  if (bs != CUBLAS_STATUS_SUCCESS) {
    h->blas = nullptr;
    return blas_fail(bs, "cublasCreate");
  }
  // emulated compute types (gemm_mode 1) are used whenever they are requested
  bs = cublasSetEmulationStrategy(h->blas, CUBLAS_EMULATION_STRATEGY_EAGER);
  if (bs != CUBLAS_STATUS_SUCCESS) return blas_fail(bs, "cublasSetEmulationStrategy");
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  *out = h.release();
  return CEED_OK;
}

extern "C" int ceed_nt_destroy(ceed_nt_t h) {
  if (!h) return CEED_OK;
  cudaDeviceSynchronize();
  NtFree()(h);
  return CEED_OK;
}

extern "C" size_t ceed_nt_qdata_bytes(ceed_nt_t h, int op, int prec) {
  if (nt_check(h, op, prec) != CEED_OK) return 0;
  return (size_t)(op == CEED_OP_MASS ? 1 : 6) * h->Q * h->Es * (prec == CEED_F32 ? 4 : 8);
}

extern "C" int ceed_nt_build_qdata(ceed_nt_t h, int op, int coeff_kind, const double *coeff, int prec, void *qdata,
                                   void *stream) {
  int st = nt_check(h, op, prec);
  if (st != CEED_OK) return st;
  if (!qdata) return fail(CEED_ERR_INVALID, "null qdata");
  double cconst = 1.0;
  if (coeff_kind == CEED_COEFF_CONST) {
    if (!coeff || !(coeff[0] > 0.0)) return fail(CEED_ERR_INVALID, "CONST coefficient needs a positive host value");
    cconst = coeff[0];
  } else if (coeff_kind == CEED_COEFF_PER_QPT) {
    if (!coeff) return fail(CEED_ERR_INVALID, "PER_QPT coefficient needs a device array");
  } else if (coeff_kind != CEED_COEFF_ONE && coeff_kind != CEED_COEFF_SINE) {
    return fail(CEED_ERR_INVALID, "unknown coefficient kind");
  }
  cudaStream_t s = (cudaStream_t)stream;
  CEED_CUDA_CHECK(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  const int64_t tot = (int64_t)h->Q * h->Es;
  const unsigned grid = (unsigned)((tot + 255) / 256);
  if (prec == CEED_F64)
    nt_qdata_kernel<double><<<grid, 256, 0, s>>>(h->E, h->Es, h->Q, op, h->d_vert, h->d_qw, h->d_qref, coeff_kind, cconst,
                                                 coeff, static_cast<double *>(qdata), h->d_err);
  else if (prec == CEED_F64_DF)
    nt_qdata_kernel<DF><<<grid, 256, 0, s>>>(h->E, h->Es, h->Q, op, h->d_vert, h->d_qw, h->d_qref, coeff_kind, cconst,
                                             coeff, static_cast<DF *>(qdata), h->d_err);
  else
    nt_qdata_kernel<float><<<grid, 256, 0, s>>>(h->E, h->Es, h->Q, op, h->d_vert, h->d_qw, h->d_qref, coeff_kind, cconst,
                                                coeff, static_cast<float *>(qdata), h->d_err);
  CEED_CUDA_CHECK(cudaGetLastError());
  int err = 0;
  CEED_CUDA_CHECK(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  if (err == CEED_ERR_BAD_GEOMETRY) return fail(CEED_ERR_BAD_GEOMETRY, "det J <= 0 in some simplex");
  return CEED_OK;
}

extern "C" int ceed_nt_apply(ceed_nt_t h, int op, const void *qdata, int prec, const double *x, double *y,
                             unsigned flags, void *stream) {
  int st = nt_check(h, op, prec);
  if (st != CEED_OK) return st;
  if (!qdata || !x || !y) return fail(CEED_ERR_INVALID, "null qdata, x or y");
  if (x == y) return fail(CEED_ERR_INVALID, "x and y must not overlap");
  return nt_apply(h, op, qdata, prec, x, y, flags, h->choice[op][nt_slot(prec)], (cudaStream_t)stream);
}

static int nt_check_choice(ceed_nt_t h, int prec, int algo, int64_t eta, int gemm_mode) {
  if (algo != CEED_NT_FUSED && algo != CEED_NT_GEMM && algo != CEED_NT_TC)
    return fail(CEED_ERR_INVALID, "algo must be FUSED, GEMM or TC");
  if (prec == CEED_F64_DF && algo != CEED_NT_FUSED)
    return fail(CEED_ERR_INVALID, "the double-float precision has the fused algorithm only");
  if (algo == CEED_NT_TC) {
    if (prec != CEED_F32) return fail(CEED_ERR_INVALID, "the tensor-core algorithm computes in FP32 (prec F32)");
    if (!nt_tc_supported(h->P)) return fail(CEED_ERR_UNSUPPORTED, "tensor-core algorithm: P must be 4, 10, 20, 35, 56 or 84");
  }
  if (algo == CEED_NT_GEMM) {
    if (eta < 0) return fail(CEED_ERR_INVALID, "eta must be >= 0");
    if (gemm_mode < 0 || gemm_mode > 2 || (gemm_mode == 2 && prec != CEED_F32))
      return fail(CEED_ERR_INVALID, "gemm_mode: 0 native, 1 emulated, 2 TF32 (F32 only)");
  }
  return CEED_OK;
}

extern "C" int ceed_nt_set_algorithm(ceed_nt_t h, int op, int prec, int algo, int64_t eta, int gemm_mode) {
  int st = nt_check(h, op, prec);
  if (st != CEED_OK) return st;
  if ((st = nt_check_choice(h, prec, algo, eta, gemm_mode)) != CEED_OK) return st;
  if (algo == CEED_NT_GEMM && (st = nt_ensure_gemm_workspace(h)) != CEED_OK) return st;
  if (algo == CEED_NT_TC && (st = nt_tc_prepare(h)) != CEED_OK) return st;
  NtChoice &c = h->choice[op][nt_slot(prec)];
  c.algo = algo;
  c.eta = algo == CEED_NT_GEMM ? eta : 0;
  c.gemm_mode = algo == CEED_NT_GEMM ? gemm_mode : 0;
  c.ms = 0.f;
  return CEED_OK;
}

extern "C" int ceed_nt_get_algorithm(ceed_nt_t h, int op, int prec, int32_t *algo, int64_t *eta, int32_t *gemm_mode,
                                     float *ms) {
  int st = nt_check(h, op, prec);
  if (st != CEED_OK) return st;
  const NtChoice &c = h->choice[op][nt_slot(prec)];
  if (algo) *algo = c.algo;
  if (eta) *eta = c.eta;
  if (gemm_mode) *gemm_mode = c.gemm_mode;
  if (ms) *ms = c.ms;
  return CEED_OK;
}

extern "C" int ceed_nt_autotune(ceed_nt_t h, int op, const void *qdata, int prec, const double *x, double *y,
                                int include_tf32, void *stream) {
  int st = nt_check(h, op, prec);
  if (st != CEED_OK) return st;
  if (!qdata || !x || !y || x == y) return fail(CEED_ERR_INVALID, "null or overlapping qdata, x, y");
  if ((st = nt_ensure_gemm_workspace(h)) != CEED_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<NtChoice> cand;
  cand.push_back(NtChoice());
  if (prec == CEED_F32 && nt_tc_supported(h->P)) {
    if ((st = nt_tc_prepare(h)) != CEED_OK) return st;
    NtChoice c;
    c.algo = CEED_NT_TC;
    cand.push_back(c);
  }
  const int64_t etas[] = {0, 1024, 4096, 16384, 65536};
  // the double-float precision has the fused algorithm only
  const int nmodes = prec == CEED_F64_DF ? 0 : (prec == CEED_F32 && include_tf32) ? 3 : 2;
  for (int mode = 0; mode < nmodes; ++mode)
    for (int64_t eta : etas) {
      if (eta != 0 && eta >= h->E) continue;
      NtChoice c;
      c.algo = CEED_NT_GEMM;
      c.eta = eta;
      c.gemm_mode = mode;
      cand.push_back(c);
    }
  cudaEvent_t e0, e1;
  CEED_CUDA_CHECK(cudaEventCreate(&e0));
  CEED_CUDA_CHECK(cudaEventCreate(&e1));
  NtChoice best;
  best.ms = 1e30f;
  for (NtChoice &c : cand) {
    for (int w = 0; w < 2; ++w)
      if ((st = nt_apply(h, op, qdata, prec, x, y, 0, c, s)) != CEED_OK) break;
    if (st != CEED_OK) break;
    const int reps = 5;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == CEED_OK; ++r) st = nt_apply(h, op, qdata, prec, x, y, 0, c, s);
    cudaEventRecord(e1, s);
    if (st != CEED_OK) break;
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      st = cuda_fail(ce, "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c.ms = ms / reps;
    if (c.ms < best.ms) best = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CEED_OK) return st;
  h->choice[op][nt_slot(prec)] = best;
  return CEED_OK;
}

extern "C" int ceed_nt_status(ceed_nt_t h, void *stream) {
  if (!h) return fail(CEED_ERR_INVALID, "null non-tensor operator handle");
  int err = 0;
  CEED_CUDA_CHECK(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CEED_CUDA_CHECK(cudaStreamSynchronize((cudaStream_t)stream));
  if (err == CEED_ERR_TIMEOUT) return fail(CEED_ERR_TIMEOUT, "a bounded device wait of the tensor-core kernel expired");
  return CEED_OK;
}
