// Device helpers shared by the setup and adjoint kernels: trilinear element map, adjugate,
// analytic coefficient and manufactured source.
#pragma once

#include "internal.h"

namespace ceedgb {

// x(r, s, t) = sum_v N_v X_v with N_v = (1 +- r)(1 +- s)(1 +- t) / 8 (vertex v = vx + 2 vy + 4 vz),
// and J[a][b] = dx_a / dr_b.
__device__ __forceinline__ void trilinear_map(const double *__restrict__ V, double r, double s, double t,
                                              double X[3], double J[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    X[a] = 0.0;
    J[a][0] = J[a][1] = J[a][2] = 0.0;
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double sr = (v & 1) ? 1.0 : -1.0, ss = (v & 2) ? 1.0 : -1.0, st = (v & 4) ? 1.0 : -1.0;
    const double fr = 0.5 * (1.0 + sr * r), fs = 0.5 * (1.0 + ss * s), ft = 0.5 * (1.0 + st * t);
    const double N = fr * fs * ft;
    const double dr = 0.5 * sr * fs * ft, ds = 0.5 * ss * fr * ft, dt = 0.5 * st * fr * fs;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double xv = V[v * 3 + a];
      X[a] += N * xv;
      J[a][0] += dr * xv;
      J[a][1] += ds * xv;
      J[a][2] += dt * xv;
    }
  }
}

// adj(J) (so that J adj(J) = det(J) I); returns det(J).
__device__ __forceinline__ double adjugate(const double J[3][3], double A[3][3]) {
  A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

// k(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)
__device__ __forceinline__ double sine_coefficient(const double X[3]) {
  return 1.0 + 0.5 * sinpi(2.0 * X[0]) * sinpi(2.0 * X[1]) * sinpi(2.0 * X[2]);
}

// f = -div(k grad u*) for u* = sin(pi x) sin(pi y) sin(pi z):
// f = 3 pi^2 k u* - grad k . grad u*  (k = 1 when coeff_kind is ONE).
__device__ __forceinline__ double manufactured_source(const double X[3], int coeff_kind) {
  const double pi = 3.14159265358979323846;
  const double sx = sinpi(X[0]), sy = sinpi(X[1]), sz = sinpi(X[2]);
  const double cx = cospi(X[0]), cy = cospi(X[1]), cz = cospi(X[2]);
  const double u = sx * sy * sz;
  if (coeff_kind != CEED_COEFF_SINE) return 3.0 * pi * pi * u;
  const double s2x = sinpi(2.0 * X[0]), s2y = sinpi(2.0 * X[1]), s2z = sinpi(2.0 * X[2]);
  const double c2x = cospi(2.0 * X[0]), c2y = cospi(2.0 * X[1]), c2z = cospi(2.0 * X[2]);
  const double k = 1.0 + 0.5 * s2x * s2y * s2z;
  const double gk_dot_gu = pi * pi * (c2x * s2y * s2z * cx * sy * sz + s2x * c2y * s2z * sx * cy * sz +
                                      s2x * s2y * c2z * sx * sy * cz);
  return 3.0 * pi * pi * k * u - gk_dot_gu;
}

// ------------------------------------------------------------------ curved (isoparametric) geometry
// x(xi) = sum_n phi_n(xi) x_n with the element's own Q_p basis: X and J at the quadrature points by
// sum factorization of the gathered node positions, one coordinate at a time (passes along r, s,
// t with the 1D interpolation B[q][a] and the derivative of the nodal basis G[q][a] at the points).
struct IsoTab {
  double B[MAX_Q * MAX_P];  // l_a(x_q)
  double G[MAX_Q * MAX_P];  // l_a'(x_q)
};

constexpr int ISO_THREADS = 256;
constexpr int ISO_PPT = (MAX_Q * MAX_Q * MAX_Q + ISO_THREADS - 1) / ISO_THREADS;  // points per thread

// shared memory (doubles): node values P^3, r pass 2 P^2 Q, s pass 3 P Q^2
__host__ __device__ inline int iso_smem_doubles(int P, int Q) { return P * P * P + 2 * P * P * Q + 3 * P * Q * Q; }

// X[t][c] and J[t][c][b] = dx_c / dxi_b at points q = threadIdx.x + t * blockDim.x (q < Q^3) of one
// element whose node indices (restriction with flags) are emap_e; blockDim.x * ISO_PPT >= Q^3.
__device__ inline void iso_geometry(const double *__restrict__ coords, const uint32_t *__restrict__ emap_e, int P,
                                    int Q, const IsoTab &T, double *sm, double X[ISO_PPT][3],
                                    double J[ISO_PPT][3][3]) {
  const int nd = P * P * P, nq = Q * Q * Q;
  double *s0 = sm, *s1b = s0 + nd, *s1d = s1b + P * P * Q;
  double *s2bb = s1d + P * P * Q, *s2bd = s2bb + P * Q * Q, *s2db = s2bd + P * Q * Q;
#pragma unroll
  for (int c = 0; c < 3; ++c) {  // unrolled: X and J stay in registers
    for (int n = threadIdx.x; n < nd; n += blockDim.x) s0[n] = coords[(int64_t)(emap_e[n] & DOF_MASK) * 3 + c];
    __syncthreads();
    for (int o = threadIdx.x; o < P * P * Q; o += blockDim.x) {  // r: (cc, b, i)
      const int i = o % Q, b = (o / Q) % P, cc = o / (Q * P);
      double vb = 0.0, vd = 0.0;
      for (int a = 0; a < P; ++a) {
        const double x = s0[(cc * P + b) * P + a];
        vb += T.B[i * P + a] * x;
        vd += T.G[i * P + a] * x;
      }
      s1b[o] = vb;
      s1d[o] = vd;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < P * Q * Q; o += blockDim.x) {  // s: (cc, j, i)
      const int i = o % Q, j = (o / Q) % Q, cc = o / (Q * Q);
      double bb = 0.0, bd = 0.0, db = 0.0;
      for (int b = 0; b < P; ++b) {
        const double u = s1b[(cc * P + b) * Q + i], ud = s1d[(cc * P + b) * Q + i];
        bb += T.B[j * P + b] * u;
        bd += T.G[j * P + b] * u;
        db += T.B[j * P + b] * ud;
      }
      s2bb[o] = bb;
      s2bd[o] = bd;
      s2db[o] = db;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < ISO_PPT; ++t) {  // t: my points
      const int q = threadIdx.x + t * blockDim.x;
      if (q >= nq) continue;
      const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
      double x = 0.0, jr = 0.0, js = 0.0, jt = 0.0;
      for (int cc = 0; cc < P; ++cc) {
        const int o = (cc * Q + j) * Q + i;
        x += T.B[k * P + cc] * s2bb[o];
        jt += T.G[k * P + cc] * s2bb[o];
        js += T.B[k * P + cc] * s2bd[o];
        jr += T.B[k * P + cc] * s2db[o];
      }
      X[t][c] = x;
      J[t][c][0] = jr;
      J[t][c][1] = js;
      J[t][c][2] = jt;
    }
    __syncthreads();  // s0 is refilled by the next coordinate
  }
}

}  // namespace ceedgb
