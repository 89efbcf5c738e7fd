// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ceed_gb300.h"
#include "df.cuh"

namespace ceedgb {

constexpr int MAX_P = 9;    // nodes per direction (p = 8)
constexpr int MAX_Q = 10;   // quadrature points per direction (Gauss, p = 8)

// Restriction entries: low 29 bits are the L-vector node; bit 31 marks the first element (in
// colour order) that writes the node, bit 29 the last one, bit 30 a Dirichlet node.
constexpr uint32_t FLAG_FIRST = 1u << 31;
constexpr uint32_t FLAG_DIR = 1u << 30;
constexpr uint32_t FLAG_LAST = 1u << 29;
constexpr uint32_t DOF_MASK = (1u << 29) - 1u;

// Brick flags (brick.cuh): bits 0-2 parity of the brick's lattice coordinates (x, y, z); bits 3-8 set
// when the brick's face at -x, +x, -y, +y, -z, +z touches another brick.
constexpr uint32_t BRICK_MX = 1u << 3, BRICK_PX = 1u << 4, BRICK_MY = 1u << 5, BRICK_PY = 1u << 6;
constexpr uint32_t BRICK_MZ = 1u << 7, BRICK_PZ = 1u << 8;
constexpr uint32_t BRICK_DIR = 1u << 9;  // some node of the brick is a Dirichlet node
// Elements of a brick along z (2 x 2 x BRICK_KZ elements per brick).  One layer: 2 x 2 x 2 bricks
// read about 6% fewer nodes but fit half as many blocks per SM, and measured slower.
constexpr int BRICK_KZ = 1;

// Even-odd split of a centro-(anti)symmetric NO x NI matrix M (M[NO-1-i][NI-1-j] = +-M[i][j]):
// E/O are the (NO/2) x (NI/2) blocks acting on folded inputs, cmid the middle input column
// (odd NI), rmid the middle output row (odd NO), cc the centre entry.
constexpr int EO_H = 5;
template <typename T>
struct EOMat {
  T E[EO_H * EO_H];
  T O[EO_H * EO_H];
  T cmid[EO_H];
  T rmid[EO_H];
  T cc;
};

// Double-float form of the even-odd blocks, laid out for packed two-lane FP32 arithmetic: entry k
// of the E block and entry k of the O block side by side (lane 0 = E, lane 1 = O), high words in
// eo_hi and low words in eo_lo; same size as the generic layout.
template <>
struct EOMat<DF> {
  float2 eo_hi[EO_H * EO_H];
  float2 eo_lo[EO_H * EO_H];
  DF cmid[EO_H];
  DF rmid[EO_H];
  DF cc;
};
static_assert(sizeof(EOMat<DF>) == sizeof(EOMat<double>), "double-float even-odd blocks: layout size");

// 1D operators passed to kernels by value (kernel parameters live in the constant bank, so
// compile-time indices become constant operands of the FMAs).
template <typename T>
struct OpTab {
  T B[MAX_Q * MAX_P];   // B[q * P + a] = l_a(xi_q): GLL Lagrange basis at the quadrature points
  T D[MAX_Q * MAX_Q];   // D[i * Q + m] = derivative at xi_i of the Lagrange basis on the Q points
  EOMat<T> eB, eBT, eD, eDT;  // even-odd forms of B (Q x P), B^T, D (Q x Q), D^T
  T qx[MAX_Q];                 // quadrature points (reference coordinates)
};

// Internal operator id of the diffusion operator whose geometric factors are recomputed from the
// trilinear map at every application (quadrature data: 24 map coefficients + w k per point).
constexpr int OP_DIFF_GEO = 2;
constexpr int GEO_COEFFS = 24;   // a1..a7 (21 floats) + 3 pad

// Quadrature data layout: [colour-sorted element][component][Q^3], each element block padded to a
// multiple of 16 bytes so that it can be moved by one TMA bulk copy.
__host__ __device__ inline int64_t qdata_estride(int op, size_t elem_bytes, int Q) {
  const int64_t n = (op == CEED_OP_DIFFUSION) ? 6 * Q * Q * Q : (op == OP_DIFF_GEO) ? GEO_COEFFS + Q * Q * Q : Q * Q * Q;
  const int64_t b = n * (int64_t)elem_bytes;
  return ((b + 15) / 16) * 16 / (int64_t)elem_bytes;
}

// Bounded device waits: polls of a TMA copy's mbarrier, and of the persistent batched launch's grid
// barrier, before the kernel gives up and records CEED_ERR_TIMEOUT.  ceed_set_wait_limits overrides
// both (process-wide, for launches issued afterwards) so that tests can make the waits run out.
constexpr int WAIT_COPY_DEFAULT = 1 << 22;
constexpr long long WAIT_GRID_DEFAULT = 1LL << 25;
int copy_wait_limit();
long long grid_wait_limit();

// Device-resident scalars of a CG run (the host reads them between batches of iterations).
struct CgScalars {
  double rz, rz_new, pq, alpha, beta, rr, bb, tol2;
  double rr_out, bb_out;
  int done, iters, nonfinite, timeout;  // timeout: a grid barrier of the fused iteration gave up
};

struct QRule {
  double x[MAX_Q];
  double w[MAX_Q];
};

// Apply-kernel variant: elements per thread block, and whether quadrature data is staged in
// shared memory by a TMA bulk copy (1) or read from global memory at the pointwise step (0); stage 2
// and 3 select the brick kernel (2 x 2 x BRICK_KZ elements per block) without and with staging.
struct ApplyChoice {
  int ne = 0;      // 0: not tuned (use the default)
  int stage = 1;
  float ms = 0.f;  // time of one application when tuned
};

}  // namespace ceedgb

namespace ceedgb {
// Launch shape of the persistent batched apply.
struct BatchLaunch {
  int threads;     // threads per block
  int stage;       // TMA staging of quadrature data
  unsigned grid;   // 0: as many blocks as are co-resident
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
  double *d_coords = nullptr;           // [n_ldof][3] curved (isoparametric) node positions, or null
  int *d_err = nullptr;                 // device status word
  bool has_dirichlet = false;
  ceedgb::OpTab<double> tab64;
  ceedgb::OpTab<float> tab32;
  ceedgb::OpTab<ceedgb::DF> tabdf;     // double-float tables of the FP64-accurate FP32-pipe operator
  ceedgb::QRule rule;                   // quadrature rule of the mesh
  double gll_x[ceedgb::MAX_P];          // GLL nodes of the basis
  ceedgb::ApplyChoice tuned[3][6];      // [op][prec] autotuned apply variant
  // 2 x 2 x BRICK_KZ element bricks of a structured lattice (brick.cuh), found at setup; n_bricks = 0
  // if the mesh is not such a lattice
  int64_t n_bricks = 0;
  std::vector<int64_t> brick_start;     // brick ranges of the 8 brick colours, size 9
  int64_t brick_sy = 0, brick_sz = 0;   // node-lattice strides
  int32_t *d_gbase = nullptr;           // [brick] corner node
  int32_t *d_gelem = nullptr;           // [brick][4 BRICK_KZ] colour-sorted elements
  uint32_t *d_gflags = nullptr;         // [brick] parity and neighbour bits
  uint32_t *d_dirbits = nullptr;        // Dirichlet bit per node (meshes with a Dirichlet mask)
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
// Raises the dynamic shared-memory limit of kernel `func` to at least `bytes` on the current device
// (the opt-in is a per-context attribute), once per (kernel, device, size); thread-safe.
int ensure_dynamic_smem(const void *func, size_t bytes);
int nq_of(const ceed_mesh_t m);
size_t prec_size(int prec);

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
  int ne = 0;        // > 0: force this many elements per block (autotuner), else tuned/default
  int stage = 1;     // with ne > 0: staging switch
  double *dot_part = nullptr;  // non-null (ncol = 1): per-block partial sums of x . y over final node values
  int64_t *dot_n = nullptr;    // out: number of partial sums written
};
int launch_apply_f64(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_f32(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_qf32geo(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_df(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);

// overlapping Schwarz smoother (schwarz.cu)
int launch_schwarz(ceed_schwarz_t sw, const double *r, double *z, int masked, cudaStream_t s);

// p-multigrid transfers (pmg_kernels.cu)
int check_transfer_pair(ceed_mesh_t coarse, ceed_mesh_t fine);
int launch_prolong(ceed_mesh_t coarse, ceed_mesh_t fine, const double *uc, double *uf, int add, cudaStream_t s);
int launch_restrict(ceed_mesh_t coarse, ceed_mesh_t fine, const double *rf, double *rc, cudaStream_t s);

}  // namespace ceedgb
