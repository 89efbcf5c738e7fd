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

}  // namespace ceedgb
