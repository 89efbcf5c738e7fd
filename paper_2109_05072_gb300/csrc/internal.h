// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ceed_gb300.h"

namespace ceedgb {

constexpr int MAX_P = 9;    // nodes per direction (p = 8)
constexpr int MAX_Q = 10;   // quadrature points per direction (Gauss, p = 8)

// Restriction entries: low 30 bits are the L-vector node; bit 31 marks the first element (in
// colour order) that writes the node, bit 30 a Dirichlet node.
constexpr uint32_t FLAG_FIRST = 1u << 31;
constexpr uint32_t FLAG_DIR = 1u << 30;
constexpr uint32_t DOF_MASK = (1u << 30) - 1u;

// 1D operators passed to kernels by value (kernel parameters live in the constant bank, so
// compile-time indices become constant operands of the FMAs).
template <typename T>
struct OpTab {
  T B[MAX_Q * MAX_P];   // B[q * P + a] = l_a(xi_q): GLL Lagrange basis at the quadrature points
  T D[MAX_Q * MAX_Q];   // D[i * Q + m] = derivative at xi_i of the Lagrange basis on the Q points
};

struct QRule {
  double x[MAX_Q];
  double w[MAX_Q];
};

}  // namespace ceedgb

struct ceed_mesh_s {
  int device = 0;
  int64_t E = 0, n_ldof = 0;
  int p = 0, P = 0, Q = 0, q_rule = 0, ncomp = 1;
  int n_colors = 0;
  std::vector<int64_t> color_start;     // sorted positions, size n_colors + 1
  uint32_t *d_emap = nullptr;           // [E][P^3] colour-sorted restriction with flags
  int32_t *d_perm = nullptr;            // sorted position -> caller's element index
  double *d_vertices = nullptr;         // [E][8][3] colour-sorted
  int *d_err = nullptr;                 // device status word
  bool has_dirichlet = false;
  ceedgb::OpTab<double> tab64;
  ceedgb::OpTab<float> tab32;
  ceedgb::QRule rule;                   // quadrature rule of the mesh
  double gll_x[ceedgb::MAX_P];          // GLL nodes of the basis
};

namespace ceedgb {

// error reporting (thread-local message)
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);
#define CEED_CUDA_CHECK(call)                                   \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return ::ceedgb::cuda_fail(_e, #call); \
  } while (0)

int check_mesh(ceed_mesh_t m);
int nq_of(const ceed_mesh_t m);

// host-side 1D bases (mesh.cu)
void gll_rule(int n, double *x, double *w);
void gauss_rule(int n, double *x, double *w);

// apply launchers: one launch per colour on `stream`
struct ApplyReq {
  int op;            // ceed_op
  int prec;          // ceed_prec of qdata
  const void *qdata;
  const double *x;
  double *y;
  int ncol;          // ncomp * nrhs
  int masked;
};
int launch_apply_f64(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_f32(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);

}  // namespace ceedgb
