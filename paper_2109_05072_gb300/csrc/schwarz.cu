// Overlapping Schwarz smoother with fast diagonalization (Lottes and Fischer, "Hybrid
// multigrid/Schwarz algorithms for the spectral element method", J. Sci. Comput. 24, 2005): the
// Schwarz/fast-diagonalization preconditioning the paper lists beside p-multigrid (Section 1),
// built on the same per-element tensor passes as the operator.
//
// Each element's local problem lives on its own GLL nodes with Dirichlet conditions one node into
// each neighbour (minimal overlap).  Its operator is replaced by the separable operator of a box
// with the element's mean side lengths h and mean coefficient k,
//   A_e = k (B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x + A_z (x) B_y (x) B_x),
// A_d = (2/h_d) A^, B_d = (h_d/2) B^, (A^, B^) the GLL stiffness and mass of three reference
// elements assembled side by side and restricted to the middle one.  Fast diagonalization inverts
// it: with A^ S = B^ S L, S^T B^ S = I,
//   A_e^{-1} = (2/h_x)(2/h_y)(2/h_z) / k (S (x) S (x) S) diag(1 / sum_d (2/h_d)^2 L) (S (x) S (x) S)^T.
// The smoother is z = sum_e R_e^T W A_e^{-1} W R_e r with W = multiplicity^{-1/2} (symmetric).
// One kernel per colour: gather, three transposed 1D passes, diagonal scaling, three 1D passes,
// scatter in colour order (no two elements of a colour share a node: no atomics, deterministic).
// Arithmetic in FP32 (a preconditioner), L-vectors FP64.
#include <cmath>
#include <memory>
#include <new>
#include <vector>

#include "convert.cuh"
#include "geometry.cuh"
#include "internal.h"

namespace ceedgb {

struct SchwarzTab {
  float S[MAX_P * MAX_P];   // S[a * P + i]: eigenvector i at node a
  float lam[MAX_P];
};

}  // namespace ceedgb

struct ceed_schwarz_s {
  ceed_mesh_t mesh = nullptr;
  float4 *d_geo = nullptr;   // per colour-sorted element: (2/h_x, 2/h_y, 2/h_z, 1/k)
  float *d_w = nullptr;      // [n_ldof] multiplicity^{-1/2}
  ceedgb::SchwarzTab tab;
};

namespace ceedgb {
namespace {

// Symmetric eigendecomposition C = V diag(d) V^T by cyclic Jacobi rotations (small n).
void jacobi_eig(int n, std::vector<double> C, std::vector<double> &V, std::vector<double> &d) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += C[i * n + j] * C[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = C[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (C[q * n + q] - C[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // C <- J^T C J
          const double ckp = C[k * n + p], ckq = C[k * n + q];
          C[k * n + p] = c * ckp - s * ckq;
          C[k * n + q] = s * ckp + c * ckq;
        }
        for (int k = 0; k < n; ++k) {
          const double cpk = C[p * n + k], cqk = C[q * n + k];
          C[p * n + k] = c * cpk - s * cqk;
          C[q * n + k] = s * cpk + c * cqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  d.resize(n);
  for (int i = 0; i < n; ++i) d[i] = C[i * n + i];
}

// The 1D fast-diagonalization basis of order p = P - 1 on GLL nodes, in FP64: S[a * P + i] is
// eigenvector i at node a, lam[i] its eigenvalue.
void fdm_1d(int P, double *S_out, double *lam_out) {
  double x[MAX_P], w[MAX_P];
  gll_rule(P, x, w);
  // differentiation matrix D[q][j] = l_j'(x_q) of the Lagrange basis on the GLL nodes
  double c[MAX_P], D[MAX_P * MAX_P];
  for (int i = 0; i < P; ++i) {
    c[i] = 1.0;
    for (int k = 0; k < P; ++k)
      if (k != i) c[i] *= x[i] - x[k];
  }
  for (int q = 0; q < P; ++q)
    for (int j = 0; j < P; ++j) {
      if (q != j) {
        D[q * P + j] = c[q] / (c[j] * (x[q] - x[j]));
      } else {
        double s = 0.0;
        for (int k = 0; k < P; ++k)
          if (k != q) s += 1.0 / (x[q] - x[k]);
        D[q * P + j] = s;
      }
    }
  // element stiffness K = D^T diag(w) D; three elements assembled, restricted to the middle one
  std::vector<double> A(P * P, 0.0), B(P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double s = 0.0;
      for (int q = 0; q < P; ++q) s += w[q] * D[q * P + i] * D[q * P + j];
      A[i * P + j] = s;
    }
  const int p = P - 1;
  const double k00 = A[0], kpp = A[p * P + p];
  A[0] += kpp;               // the left neighbour's last node is this element's first
  A[p * P + p] += k00;       // the right neighbour's first node is this element's last
  for (int i = 0; i < P; ++i) B[i] = w[i];
  B[0] += w[p];
  B[p] += w[0];
  // generalized problem A S = B S L through C = B^{-1/2} A B^{-1/2} = V L V^T, S = B^{-1/2} V
  std::vector<double> C(P * P), V, lam;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) C[i * P + j] = A[i * P + j] / std::sqrt(B[i] * B[j]);
  jacobi_eig(P, C, V, lam);
  for (int a = 0; a < P; ++a)
    for (int i = 0; i < P; ++i) S_out[a * P + i] = V[a * P + i] / std::sqrt(B[a]);
  for (int i = 0; i < P; ++i) lam_out[i] = lam[i];
}

// The kernel's FP32 copy of the tables.
void fdm_tables(int P, SchwarzTab &tab) {
  double S[MAX_P * MAX_P], lam[MAX_P];
  fdm_1d(P, S, lam);
  for (int k = 0; k < P * P; ++k) tab.S[k] = (float)S[k];
  for (int i = 0; i < P; ++i) tab.lam[i] = (float)lam[i];
}

// per colour-sorted element: mean side lengths (four edges along each reference axis) and mean
// coefficient over the GLL nodes of the trilinear map
__global__ void schwarz_geo_kernel(int64_t E, int P, const double *__restrict__ vert, int coeff_kind, double cconst,
                                   QRule gl, float4 *__restrict__ geo) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= E) return;
  const double *V = vert + s * 24;
  double h[3];
  for (int d = 0; d < 3; ++d) {
    double acc = 0.0;
    for (int v = 0; v < 8; ++v) {
      if ((v >> d) & 1) continue;
      const int u = v | (1 << d);
      double dx = 0.0;
      for (int a = 0; a < 3; ++a) dx += (V[u * 3 + a] - V[v * 3 + a]) * (V[u * 3 + a] - V[v * 3 + a]);
      acc += sqrt(dx);
    }
    h[d] = 0.25 * acc;
  }
  double k = 1.0;
  if (coeff_kind == CEED_COEFF_CONST) {
    k = cconst;
  } else if (coeff_kind == CEED_COEFF_SINE) {
    double acc = 0.0;
    for (int c = 0; c < P; ++c)
      for (int b = 0; b < P; ++b)
        for (int a = 0; a < P; ++a) {
          double X[3], J[3][3];
          trilinear_map(V, gl.x[a], gl.x[b], gl.x[c], X, J);
          acc += sine_coefficient(X);
        }
    k = acc / ((double)P * P * P);
  }
  geo[s] = make_float4((float)(2.0 / h[0]), (float)(2.0 / h[1]), (float)(2.0 / h[2]), (float)(1.0 / k));
}

__global__ void count_kernel(int64_t n, const uint32_t *__restrict__ emap, float *__restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[emap[i] & DOF_MASK], 1.0f);
}

__global__ void rsqrt_kernel(int64_t n, float *__restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = w[i] > 0.f ? rsqrtf(w[i]) : 0.f;
}

// One colour: NE elements per block, P^2 threads per element (one per line of the element).
template <int P>
__global__ void schwarz_kernel(int64_t s0, int64_t ne, const uint32_t *__restrict__ emap,
                               const double *__restrict__ r, double *__restrict__ z, const float4 *__restrict__ geo,
                               const float *__restrict__ w, SchwarzTab tab, int masked) {
  constexpr int L = P * P, N = P * P * P;
  constexpr int NE = L >= 128 ? 1 : 128 / L;
  __shared__ float su[NE][N], sv[NE][N];
  const int el = threadIdx.x / L, t = threadIdx.x % L;
  const int64_t e = (int64_t)blockIdx.x * NE + el;
  const bool valid = el < NE && e < ne;
  const int64_t s = s0 + e;
  float *u = su[el < NE ? el : 0], *v = sv[el < NE ? el : 0];
  const uint32_t *row = emap + s * N;
  float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
  // gather: thread t = b + P c owns the x-line (., b, c)
  if (valid) {
    g = geo[s];
    for (int a = 0; a < P; ++a) {
      const uint32_t m = row[a + t * P];
      const uint32_t d = m & DOF_MASK;
      u[a + t * P] = (masked && (m & FLAG_DIR)) ? 0.f : d2f_fast(r[d]) * w[d];
    }
  }
  __syncthreads();
  if (valid) {   // x pass (transposed): v[c][b][i] = sum_a S[a][i] u[c][b][a]
    for (int i = 0; i < P; ++i) {
      float acc = 0.f;
      for (int a = 0; a < P; ++a) acc = fmaf(tab.S[a * P + i], u[a + t * P], acc);
      v[i + t * P] = acc;
    }
  }
  __syncthreads();
  const int ti = t % P, tc = t / P;   // y pass: t = i + P c
  if (valid) {
    for (int j = 0; j < P; ++j) {
      float acc = 0.f;
      for (int b = 0; b < P; ++b) acc = fmaf(tab.S[b * P + j], v[ti + P * (b + P * tc)], acc);
      u[ti + P * (j + P * tc)] = acc;
    }
  }
  __syncthreads();
  const int tj = t / P;   // z pass and scaling: t = i + P j
  if (valid) {
    const float gx2 = g.x * g.x, gy2 = g.y * g.y, gz2 = g.z * g.z;
    for (int k = 0; k < P; ++k) {
      float acc = 0.f;
      for (int c = 0; c < P; ++c) acc = fmaf(tab.S[c * P + k], u[ti + P * (tj + P * c)], acc);
      const float den = gx2 * tab.lam[ti] + gy2 * tab.lam[tj] + gz2 * tab.lam[k];
      v[ti + P * (tj + P * k)] = acc * g.w / den;
    }
  }
  __syncthreads();
  if (valid) {   // back along z
    for (int c = 0; c < P; ++c) {
      float acc = 0.f;
      for (int k = 0; k < P; ++k) acc = fmaf(tab.S[c * P + k], v[ti + P * (tj + P * k)], acc);
      u[ti + P * (tj + P * c)] = acc;
    }
  }
  __syncthreads();
  if (valid) {   // back along y: t = i + P c
    for (int b = 0; b < P; ++b) {
      float acc = 0.f;
      for (int j = 0; j < P; ++j) acc = fmaf(tab.S[b * P + j], u[ti + P * (j + P * tc)], acc);
      v[ti + P * (b + P * tc)] = acc;
    }
  }
  __syncthreads();
  if (valid) {   // back along x and scatter: t = b + P c
    const float scale = g.x * g.y * g.z;
    for (int a = 0; a < P; ++a) {
      float acc = 0.f;
      for (int i = 0; i < P; ++i) acc = fmaf(tab.S[a * P + i], v[i + t * P], acc);
      const uint32_t m = row[a + t * P];
      const uint32_t d = m & DOF_MASK;
      const double val = (masked && (m & FLAG_DIR)) ? 0.0 : f2d_int(acc * scale * w[d]);
      z[d] = (m & FLAG_FIRST) ? val : z[d] + val;
    }
  }
}

template <int P>
int launch_schwarz_p(ceed_schwarz_t sw, const double *r, double *z, int masked, cudaStream_t s) {
  constexpr int L = P * P;
  constexpr int NE = L >= 128 ? 1 : 128 / L;
  const ceed_mesh_t m = sw->mesh;
  for (int c = 0; c < m->n_colors; ++c) {
    const int64_t s0 = m->color_start[c], ne = m->color_start[c + 1] - s0;
    if (ne == 0) continue;
    const unsigned grid = (unsigned)((ne + NE - 1) / NE);
    schwarz_kernel<P><<<grid, NE * L, 0, s>>>(s0, ne, m->d_emap, r, z, sw->d_geo, sw->d_w, sw->tab, masked);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

}  // namespace

int launch_schwarz(ceed_schwarz_t sw, const double *r, double *z, int masked, cudaStream_t s) {
  switch (sw->mesh->P) {
    case 2: return launch_schwarz_p<2>(sw, r, z, masked, s);
    case 3: return launch_schwarz_p<3>(sw, r, z, masked, s);
    case 4: return launch_schwarz_p<4>(sw, r, z, masked, s);
    case 5: return launch_schwarz_p<5>(sw, r, z, masked, s);
    case 6: return launch_schwarz_p<6>(sw, r, z, masked, s);
    case 7: return launch_schwarz_p<7>(sw, r, z, masked, s);
    case 8: return launch_schwarz_p<8>(sw, r, z, masked, s);
    case 9: return launch_schwarz_p<9>(sw, r, z, masked, s);
    default: return fail(CEED_ERR_UNSUPPORTED, "Schwarz smoother: p in 1..8");
  }
}

}  // namespace ceedgb

using namespace ceedgb;

extern "C" int ceed_schwarz_fdm_1d(int p, double *S, double *lambda) {
  if (p < 1 || p + 1 > MAX_P) return fail(CEED_ERR_INVALID, "p outside 1..8");
  if (!S || !lambda) return fail(CEED_ERR_INVALID, "null output array");
  fdm_1d(p + 1, S, lambda);
  return CEED_OK;
}

extern "C" int ceed_schwarz_create(ceed_mesh_t mesh, int coeff_kind, const double *coeff, ceed_schwarz_t *out,
                                   void *stream) {
  if (!mesh || !out) return fail(CEED_ERR_INVALID, "null mesh or output");
  *out = nullptr;
  if (mesh->q_rule != CEED_QRULE_GLL) return fail(CEED_ERR_UNSUPPORTED, "Schwarz smoother: GLL collocated meshes");
  if (mesh->ncomp != 1) return fail(CEED_ERR_UNSUPPORTED, "Schwarz smoother: one component");
  double cconst = 1.0;
  if (coeff_kind == CEED_COEFF_CONST) {
    if (!coeff || !(coeff[0] > 0.0)) return fail(CEED_ERR_INVALID, "CONST coefficient needs a positive host value");
    cconst = coeff[0];
  } else if (coeff_kind != CEED_COEFF_ONE && coeff_kind != CEED_COEFF_SINE) {
    return fail(CEED_ERR_UNSUPPORTED, "Schwarz smoother: coefficient ONE, CONST or SINE");
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<ceed_schwarz_s> sw(new (std::nothrow) ceed_schwarz_s());
  if (!sw) return fail(CEED_ERR_OOM, "host allocation");
  sw->mesh = mesh;
  fdm_tables(mesh->P, sw->tab);
  const int64_t E = mesh->E, n = mesh->n_ldof, nent = E * (int64_t)mesh->P * mesh->P * mesh->P;
  CEED_CUDA_CHECK(cudaMalloc(&sw->d_geo, E * sizeof(float4)));
  cudaError_t ce = cudaMalloc(&sw->d_w, n * sizeof(float));
  if (ce != cudaSuccess) {
    cudaFree(sw->d_geo);
    return cuda_fail(ce, "cudaMalloc (Schwarz weights)");
  }
  QRule gl{};
  double wq[MAX_P];
  gll_rule(mesh->P, gl.x, wq);
  schwarz_geo_kernel<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(E, mesh->P, mesh->d_vertices, coeff_kind, cconst, gl,
                                                                   sw->d_geo);
  CEED_CUDA_CHECK(cudaMemsetAsync(sw->d_w, 0, n * sizeof(float), s));
  count_kernel<<<(unsigned)((nent + 255) / 256), 256, 0, s>>>(nent, mesh->d_emap, sw->d_w);
  rsqrt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, sw->d_w);
  CEED_CUDA_CHECK(cudaGetLastError());
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  *out = sw.release();
  return CEED_OK;
}

extern "C" int ceed_schwarz_apply(ceed_schwarz_t sw, const double *r, double *z, unsigned flags, void *stream) {
  if (!sw || !r || !z || r == z) return fail(CEED_ERR_INVALID, "null or overlapping Schwarz arguments");
  return launch_schwarz(sw, r, z, (flags & CEED_APPLY_DIRICHLET) && sw->mesh->has_dirichlet ? 1 : 0,
                        (cudaStream_t)stream);
}

extern "C" int ceed_schwarz_destroy(ceed_schwarz_t sw) {
  if (!sw) return CEED_OK;
  cudaDeviceSynchronize();
  cudaFree(sw->d_geo);
  cudaFree(sw->d_w);
  delete sw;
  return CEED_OK;
}
