// Mesh handle: 1D bases, element colouring, colour-sorted restriction; apply entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <utility>

#include "internal.h"

namespace ceedgb {

static thread_local std::string g_last_error;

int fail(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char *where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? CEED_ERR_OOM : CEED_ERR_CUDA;
}

int ensure_dynamic_smem(const void *func, size_t bytes) {
  if (bytes <= 48 * 1024) return CEED_OK;
  int dev = 0;
  CEED_CUDA_CHECK(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> raised;  // (kernel, device) -> limit set so far
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = raised[{func, dev}];
  if (bytes > cur) {
    // refuse a size the device cannot give before asking for it: a failed request would leave an
    // error for the next cudaGetLastError of an unrelated call
    int optin = 0;
    CEED_CUDA_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    CEED_CUDA_CHECK(cudaFuncGetAttributes(&fa, func));
    if (bytes + fa.sharedSizeBytes > (size_t)optin)
      return fail(CEED_ERR_UNSUPPORTED, "kernel variant needs " + std::to_string(bytes + fa.sharedSizeBytes) +
                                            " bytes of shared memory per block; the device allows " +
                                            std::to_string(optin));
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it
      return cuda_fail(e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
    }
    cur = bytes;
  }
  return CEED_OK;
}

static std::atomic<int> g_copy_wait{WAIT_COPY_DEFAULT};
static std::atomic<long long> g_grid_wait{WAIT_GRID_DEFAULT};
int copy_wait_limit() { return g_copy_wait.load(std::memory_order_relaxed); }
long long grid_wait_limit() { return g_grid_wait.load(std::memory_order_relaxed); }

int check_mesh(ceed_mesh_t m) {
  if (!m) return fail(CEED_ERR_INVALID, "null mesh handle");
  return CEED_OK;
}

int nq_of(const ceed_mesh_t m) { return m->Q * m->Q * m->Q; }

// ---------------------------------------------------------------------------------------------
// 1D rules.  Legendre P_n and derivatives by the three-term recurrence; Newton iteration for
// the roots.  Gauss: roots of P_n, w = 2 / ((1 - x^2) P_n'^2).  Gauss-Lobatto: +-1 and the roots
// of P_{n-1}', w = 2 / (n (n - 1) P_{n-1}^2).
static void legendre_eval(int n, double x, double *p, double *dp, double *d2p) {
  double p0 = 1, p1 = x, d0 = 0, d1 = 1, s0 = 0, s1 = 0;
  if (n == 0) {
    *p = 1; *dp = 0; *d2p = 0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double a = (2.0 * k + 1.0) / (k + 1.0), b = (double)k / (k + 1.0);
    const double p2 = a * x * p1 - b * p0;
    const double d2 = a * (p1 + x * d1) - b * d0;
    const double s2 = a * (2.0 * d1 + x * s1) - b * s0;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
  }
  *p = p1; *dp = d1; *d2p = s1;
}

void gauss_rule(int n, double *x, double *w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double t = -std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp, d2p;
      legendre_eval(n, t, &p, &dp, &d2p);
      const double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p, dp, d2p;
    legendre_eval(n, t, &p, &dp, &d2p);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
  // exact mirror symmetry (the even-odd kernels rely on it)
  for (int i = 0; i < n / 2; ++i) {
    x[n - 1 - i] = -x[i];
    w[n - 1 - i] = w[i];
  }
  if (n & 1) x[n / 2] = 0.0;
}

void gll_rule(int n, double *x, double *w) {
  const double pi = 3.14159265358979323846;
  const int m = n - 1;
  for (int i = 0; i < n; ++i) {
    double t = -std::cos(pi * i / m);
    if (i > 0 && i < m) {
      for (int it = 0; it < 100; ++it) {
        double p, dp, d2p;
        legendre_eval(m, t, &p, &dp, &d2p);
        const double dt = dp / d2p;
        t -= dt;
        if (std::fabs(dt) < 1e-16) break;
      }
    }
    if (i == 0) t = -1.0;
    if (i == m) t = 1.0;
    double p, dp, d2p;
    legendre_eval(m, t, &p, &dp, &d2p);
    x[i] = t;
    w[i] = 2.0 / (n * m * p * p);
  }
  for (int i = 0; i < n / 2; ++i) {
    x[n - 1 - i] = -x[i];
    w[n - 1 - i] = w[i];
  }
  if (n & 1) x[n / 2] = 0.0;
}

// Barycentric weights lambda_j = 1 / prod_{m != j} (x_j - x_m).
static void bary_weights(int n, const double *x, double *lam) {
  for (int j = 0; j < n; ++j) {
    double d = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) d *= (x[j] - x[m]);
    lam[j] = 1.0 / d;
  }
}

// Interpolation matrix B[q * n + a] = l_a(t_q) for the Lagrange basis through nodes x (barycentric form).
static void interp_matrix(int n, const double *x, int nq, const double *t, double *B) {
  double lam[MAX_Q];
  bary_weights(n, x, lam);
  for (int q = 0; q < nq; ++q) {
    int hit = -1;
    for (int a = 0; a < n; ++a)
      if (t[q] == x[a]) hit = a;
    if (hit >= 0) {
      for (int a = 0; a < n; ++a) B[q * n + a] = (a == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int a = 0; a < n; ++a) den += lam[a] / (t[q] - x[a]);
    for (int a = 0; a < n; ++a) B[q * n + a] = (lam[a] / (t[q] - x[a])) / den;
  }
}

// Collocation derivative D[i * n + j] = l_j'(x_i) for the Lagrange basis through x (barycentric
// off-diagonal entries; the diagonal makes every row sum to zero).
static void deriv_matrix(int n, const double *x, double *D) {
  double lam[MAX_Q];
  bary_weights(n, x, lam);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double v = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * n + j] = v;
      s += v;
    }
    D[i * n + i] = -s;
  }
}

// Even-odd blocks of an NO x NI matrix with M[NO-1-i][NI-1-j] = S M[i][j] (symmetry enforced:
// the blocks are built from the upper half only).
static void make_eo(const double *M, int NO, int NI, int S, EOMat<double> *d, EOMat<float> *f) {
  std::memset(d, 0, sizeof(*d));
  std::memset(f, 0, sizeof(*f));
  const int HO = NO / 2, HI = NI / 2;
  for (int i = 0; i < HO; ++i) {
    for (int j = 0; j < HI; ++j) {
      const double a = M[i * NI + j], b = M[i * NI + (NI - 1 - j)];
      d->E[i * EO_H + j] = 0.5 * (a + b);
      d->O[i * EO_H + j] = 0.5 * (a - b);
    }
    if (NI & 1) d->cmid[i] = M[i * NI + HI];
  }
  if (NO & 1) {
    for (int j = 0; j < HI; ++j) d->rmid[j] = M[HO * NI + j];
    if (NI & 1) d->cc = (S > 0) ? M[HO * NI + HI] : 0.0;
  }
  const double *src = &d->E[0];
  float *dst = &f->E[0];
  for (size_t k = 0; k < sizeof(*d) / sizeof(double); ++k) dst[k] = (float)src[k];
}

static void build_tables(ceed_mesh_s *m) {
  double w_gll[MAX_P];
  gll_rule(m->P, m->gll_x, w_gll);
  if (m->q_rule == CEED_QRULE_GLL) {
    for (int i = 0; i < m->Q; ++i) {
      m->rule.x[i] = m->gll_x[i];
      m->rule.w[i] = w_gll[i];
    }
  } else {
    gauss_rule(m->Q, m->rule.x, m->rule.w);
  }
  double B[MAX_Q * MAX_P], D[MAX_Q * MAX_Q];
  interp_matrix(m->P, m->gll_x, m->Q, m->rule.x, B);
  deriv_matrix(m->Q, m->rule.x, D);
  std::memset(&m->tab64, 0, sizeof(m->tab64));
  std::memset(&m->tab32, 0, sizeof(m->tab32));
  for (int k = 0; k < m->Q * m->P; ++k) {
    m->tab64.B[k] = B[k];
    m->tab32.B[k] = (float)B[k];
  }
  for (int k = 0; k < m->Q * m->Q; ++k) {
    m->tab64.D[k] = D[k];
    m->tab32.D[k] = (float)D[k];
  }
  const int P = m->P, Q = m->Q;
  double BT[MAX_P * MAX_Q], DT[MAX_Q * MAX_Q];
  for (int q = 0; q < Q; ++q)
    for (int a = 0; a < P; ++a) BT[a * Q + q] = B[q * P + a];
  for (int i = 0; i < Q; ++i)
    for (int k = 0; k < Q; ++k) DT[k * Q + i] = D[i * Q + k];
  make_eo(B, Q, P, +1, &m->tab64.eB, &m->tab32.eB);
  make_eo(BT, P, Q, +1, &m->tab64.eBT, &m->tab32.eBT);
  make_eo(D, Q, Q, -1, &m->tab64.eD, &m->tab32.eD);
  make_eo(DT, Q, Q, -1, &m->tab64.eDT, &m->tab32.eDT);
  for (int i = 0; i < Q; ++i) {
    m->tab64.qx[i] = m->rule.x[i];
    m->tab32.qx[i] = (float)m->rule.x[i];
  }
  // double-float copy of every FP64 table (same layout, each double split into hi + lo floats)
  const double *src = reinterpret_cast<const double *>(&m->tab64);
  DF *dst = reinterpret_cast<DF *>(&m->tabdf);
  static_assert(sizeof(OpTab<double>) == sizeof(OpTab<DF>), "table layouts differ");
  for (size_t k = 0; k < sizeof(OpTab<double>) / sizeof(double); ++k) dst[k] = df_from_double(src[k]);
  // the even-odd blocks of the double-float tables use their own (E, O)-interleaved layout
  const EOMat<double> *e64[4] = {&m->tab64.eB, &m->tab64.eBT, &m->tab64.eD, &m->tab64.eDT};
  EOMat<DF> *edf[4] = {&m->tabdf.eB, &m->tabdf.eBT, &m->tabdf.eD, &m->tabdf.eDT};
  for (int t = 0; t < 4; ++t) {
    for (int k = 0; k < EO_H * EO_H; ++k) {
      const DF e = df_from_double(e64[t]->E[k]), o = df_from_double(e64[t]->O[k]);
      edf[t]->eo_hi[k] = make_float2(e.hi, o.hi);
      edf[t]->eo_lo[k] = make_float2(e.lo, o.lo);
    }
    for (int k = 0; k < EO_H; ++k) {
      edf[t]->cmid[k] = df_from_double(e64[t]->cmid[k]);
      edf[t]->rmid[k] = df_from_double(e64[t]->rmid[k]);
    }
    edf[t]->cc = df_from_double(e64[t]->cc);
  }
}

int launch_apply(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_qf32(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_qbf16(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);
int launch_apply_qf16(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s);

int launch_apply_f32(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  switch (r.prec) {
    case CEED_F32: return launch_apply_qf32(m, r, s);
    case CEED_BF16: return launch_apply_qbf16(m, r, s);
    case CEED_F16: return launch_apply_qf16(m, r, s);
    default: return fail(CEED_ERR_INVALID, "unknown precision");
  }
}

int launch_apply(ceed_mesh_t m, const ApplyReq &r, cudaStream_t s) {
  if (r.prec == CEED_F64) return launch_apply_f64(m, r, s);
  if (r.prec == CEED_F64_DF) return launch_apply_df(m, r, s);
  if (r.prec == CEED_F32_GEO) {
    if (r.op != CEED_OP_DIFFUSION) return fail(CEED_ERR_UNSUPPORTED, "F32_GEO quadrature data is for diffusion");
    return launch_apply_qf32geo(m, r, s);
  }
  return launch_apply_f32(m, r, s);
}

}  // namespace ceedgb

using namespace ceedgb;

extern "C" const char *ceed_last_error(void) { return g_last_error.c_str(); }

namespace {
struct HostFree {
  void operator()(ceed_mesh_s *m) const {
    if (!m) return;
    cudaFree(m->d_emap);
    cudaFree(m->d_perm);
    cudaFree(m->d_vertices);
    cudaFree(m->d_coords);
    cudaFree(m->d_err);
    cudaFree(m->d_gbase);
    cudaFree(m->d_gelem);
    cudaFree(m->d_gflags);
    cudaFree(m->d_dirbits);
    delete m;
  }
};
}  // namespace

// Bricks of a structured lattice (brick.cuh).  The mesh qualifies when the node numbering is a
// lexicographic lattice (x fastest) and every element's nodes are base + a + b sy + c sz with
// common strides sy, sz, the element lattice dimensions are multiples of the brick's (2, 2,
// BRICK_KZ) and every lattice cell holds one element.  Bricks are sorted by colour (parity of their
// coordinates: bit 0 x, bit 1 y, bit 2 z) and then lexicographically.  Leaves n_bricks = 0 (the
// element kernel serves the mesh) when the mesh does not qualify.
static int detect_bricks(ceed_mesh_s *m, const std::vector<uint32_t> &map, const std::vector<int32_t> &perm,
                         const std::vector<uint8_t> &dir, cudaStream_t s) {
  const int P = m->P, p = m->p;
  const int64_t E = m->E, nd = (int64_t)P * P * P, nL = m->n_ldof;
  if (p < 1 || E < 8) return CEED_OK;
  const int64_t n00 = map[0];
  const int64_t sy = (int64_t)map[P] - n00, sz = (int64_t)map[(int64_t)P * P] - n00;
  if ((int64_t)map[1] - n00 != 1 || sy < P || sz < sy * P || sz % sy != 0 || nL % sz != 0) return CEED_OK;
  const int64_t nxn = sy, nyn = sz / sy, nzn = nL / sz;
  if ((nxn - 1) % p || (nyn - 1) % p || (nzn - 1) % p) return CEED_OK;
  const int64_t Nx = (nxn - 1) / p, Ny = (nyn - 1) / p, Nz = (nzn - 1) / p;
  if (Nx * Ny * Nz != E || Nx % 2 || Ny % 2 || Nz % BRICK_KZ) return CEED_OK;
  std::vector<int32_t> elem_at;
  try {
    elem_at.assign(E, -1);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation");
  }
  for (int64_t e = 0; e < E; ++e) {
    const uint32_t *row = &map[e * nd];
    const int64_t b0 = row[0];
    const int64_t X = b0 % sy, Y = (b0 / sy) % nyn, Z = b0 / sz;
    if (X % p || Y % p || Z % p || X / p >= Nx || Y / p >= Ny || Z / p >= Nz) return CEED_OK;
    for (int c = 0, n = 0; c < P; ++c)
      for (int b = 0; b < P; ++b)
        for (int a = 0; a < P; ++a, ++n)
          if ((int64_t)row[n] != b0 + a + b * sy + c * sz) return CEED_OK;
    const int64_t cell = X / p + Nx * (Y / p + Ny * (Z / p));
    if (elem_at[cell] >= 0) return CEED_OK;
    elem_at[cell] = (int32_t)e;
  }
  std::vector<int32_t> spos(E);
  for (int64_t i = 0; i < E; ++i) spos[perm[i]] = (int32_t)i;
  const int64_t Gx = Nx / 2, Gy = Ny / 2, Gz = Nz / BRICK_KZ, G = Gx * Gy * Gz;
  constexpr int NEL = 4 * BRICK_KZ;
  std::vector<int32_t> gbase, gelem;
  std::vector<uint32_t> gflags;
  std::vector<int64_t> start(9, 0);
  gbase.reserve(G);
  gelem.reserve(NEL * G);
  gflags.reserve(G);
  for (int c = 0; c < 8; ++c) {
    start[c] = (int64_t)gbase.size();
    for (int64_t gz = (c >> 2) & 1; gz < Gz; gz += 2)
      for (int64_t gy = (c >> 1) & 1; gy < Gy; gy += 2)
        for (int64_t gx = c & 1; gx < Gx; gx += 2) {
          gbase.push_back((int32_t)(2 * gx * p + 2 * gy * p * sy + BRICK_KZ * gz * p * sz));
          for (int k = 0; k < NEL; ++k) {
            const int64_t ex = 2 * gx + (k & 1), ey = 2 * gy + ((k >> 1) & 1), ez = BRICK_KZ * gz + (k >> 2);
            gelem.push_back(spos[elem_at[ex + Nx * (ey + Ny * ez)]]);
          }
          uint32_t f = (uint32_t)((gx & 1) | ((gy & 1) << 1) | ((gz & 1) << 2));
          if (gx > 0) f |= BRICK_MX;
          if (gx + 1 < Gx) f |= BRICK_PX;
          if (gy > 0) f |= BRICK_MY;
          if (gy + 1 < Gy) f |= BRICK_PY;
          if (gz > 0) f |= BRICK_MZ;
          if (gz + 1 < Gz) f |= BRICK_PZ;
          if (!dir.empty()) {  // does the brick hold a Dirichlet node?
            const int64_t b0 = 2 * gx * p + 2 * gy * p * sy + BRICK_KZ * gz * p * sz;
            bool any = false;
            for (int64_t c = 0; c <= BRICK_KZ * p && !any; ++c)
              for (int64_t b = 0; b <= 2 * p && !any; ++b)
                for (int64_t a = 0; a <= 2 * p; ++a)
                  if (dir[b0 + a + b * sy + c * sz]) {
                    any = true;
                    break;
                  }
            if (any) f |= BRICK_DIR;
          }
          gflags.push_back(f);
        }
  }
  start[8] = (int64_t)gbase.size();
  std::vector<uint32_t> bits;
  if (!dir.empty()) {
    bits.assign((nL + 31) / 32, 0u);
    for (int64_t v = 0; v < nL; ++v)
      if (dir[v]) bits[v >> 5] |= 1u << (v & 31);
  }
  CEED_CUDA_CHECK(cudaMalloc(&m->d_gbase, G * sizeof(int32_t)));
  CEED_CUDA_CHECK(cudaMalloc(&m->d_gelem, NEL * G * sizeof(int32_t)));
  CEED_CUDA_CHECK(cudaMalloc(&m->d_gflags, G * sizeof(uint32_t)));
  CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_gbase, gbase.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_gelem, gelem.data(), NEL * G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_gflags, gflags.data(), G * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  if (!bits.empty()) {
    CEED_CUDA_CHECK(cudaMalloc(&m->d_dirbits, bits.size() * sizeof(uint32_t)));
    CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_dirbits, bits.data(), bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  }
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));  // the host vectors go out of scope
  m->brick_start = start;
  m->brick_sy = sy;
  m->brick_sz = sz;
  m->n_bricks = G;
  return CEED_OK;
}

extern "C" int ceed_setup_mesh(const ceed_mesh_desc *desc, ceed_mesh_t *out, void *stream) {
  if (!desc || !out) return fail(CEED_ERR_INVALID, "null descriptor or output");
  *out = nullptr;
  if (desc->n_elem < 1 || desc->n_ldof < 1) return fail(CEED_ERR_INVALID, "n_elem and n_ldof must be >= 1");
  if (desc->n_ldof > (int64_t)DOF_MASK) return fail(CEED_ERR_INVALID, "n_ldof must be < 2^29");
  if (desc->p < 1 || desc->p > 8) return fail(CEED_ERR_INVALID, "p must be in 1..8");
  if (desc->ncomp < 1) return fail(CEED_ERR_INVALID, "ncomp must be >= 1");
  if (!desc->elem_dofs || !desc->vertices) return fail(CEED_ERR_INVALID, "elem_dofs and vertices are required");
  const int P = desc->p + 1;
  int Q = desc->n_qpts_1d;
  if (desc->q_rule == CEED_QRULE_GLL) {
    if (Q == 0) Q = P;
    if (Q != P) return fail(CEED_ERR_UNSUPPORTED, "GLL quadrature is collocated: Q must be p+1");
  } else if (desc->q_rule == CEED_QRULE_GAUSS) {
    if (Q == 0) Q = P + 1;
    if (Q != P + 1) return fail(CEED_ERR_UNSUPPORTED, "Gauss quadrature supports Q = p+2");
  } else {
    return fail(CEED_ERR_INVALID, "unknown quadrature rule");
  }
  const int64_t E = desc->n_elem, nd = (int64_t)P * P * P, nL = desc->n_ldof;
  if (E * nd >= ((int64_t)1 << 40)) return fail(CEED_ERR_INVALID, "mesh too large");
  cudaStream_t s = (cudaStream_t)stream;

  std::unique_ptr<ceed_mesh_s, HostFree> m(new (std::nothrow) ceed_mesh_s());
  if (!m) return fail(CEED_ERR_OOM, "host allocation");
  CEED_CUDA_CHECK(cudaGetDevice(&m->device));
  m->E = E;
  m->n_ldof = nL;
  m->p = desc->p;
  m->P = P;
  m->Q = Q;
  m->q_rule = desc->q_rule;
  m->ncomp = desc->ncomp;
  build_tables(m.get());

  // ---- copy the caller's arrays to the host
  std::vector<uint32_t> map;
  std::vector<double> vert;
  std::vector<uint8_t> dir;
  try {
    map.resize(E * nd);
    vert.resize(E * 24);
    if (desc->dirichlet) dir.resize(nL);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation for the mesh copy");
  }
  CEED_CUDA_CHECK(cudaMemcpyAsync(map.data(), desc->elem_dofs, E * nd * 4, cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(vert.data(), desc->vertices, E * 24 * 8, cudaMemcpyDeviceToHost, s));
  if (desc->dirichlet) CEED_CUDA_CHECK(cudaMemcpyAsync(dir.data(), desc->dirichlet, nL, cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  m->has_dirichlet = desc->dirichlet != nullptr;

  // ---- validate: in range, no repeated node inside an element, every node referenced
  std::vector<int64_t> stamp;
  try {
    stamp.assign(nL, -1);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation");
  }
  for (int64_t e = 0; e < E; ++e) {
    const uint32_t *row = &map[e * nd];
    for (int64_t n = 0; n < nd; ++n) {
      const int64_t v = (int32_t)row[n];
      if (v < 0 || v >= nL) return fail(CEED_ERR_INVALID, "elem_dofs entry out of range at element " + std::to_string(e));
      if (stamp[v] == e) return fail(CEED_ERR_INVALID, "node repeated inside element " + std::to_string(e));
      stamp[v] = e;
    }
  }
  for (int64_t v = 0; v < nL; ++v)
    if (stamp[v] < 0) return fail(CEED_ERR_INVALID, "node " + std::to_string(v) + " belongs to no element");
  std::vector<int64_t>().swap(stamp);

  // ---- greedy colouring: no two elements of one colour share a node
  std::vector<uint8_t> color(E);
  {
    std::vector<uint64_t> used;
    try {
      used.assign(nL, 0);
    } catch (...) {
      return fail(CEED_ERR_OOM, "host allocation");
    }
    int ncol = 0;
    for (int64_t e = 0; e < E; ++e) {
      const uint32_t *row = &map[e * nd];
      uint64_t forb = 0;
      for (int64_t n = 0; n < nd; ++n) forb |= used[row[n]];
      if (forb == ~0ull) return fail(CEED_ERR_UNSUPPORTED, "element colouring needs more than 64 colours");
      const int c = __builtin_ctzll(~forb);
      color[e] = (uint8_t)c;
      ncol = std::max(ncol, c + 1);
      const uint64_t bit = 1ull << c;
      for (int64_t n = 0; n < nd; ++n) used[row[n]] |= bit;
    }
    m->n_colors = ncol;
  }
  // stable counting sort by colour
  std::vector<int64_t> start(m->n_colors + 1, 0);
  for (int64_t e = 0; e < E; ++e) start[color[e] + 1]++;
  for (int c = 0; c < m->n_colors; ++c) start[c + 1] += start[c];
  m->color_start = start;
  std::vector<int32_t> perm(E);
  {
    std::vector<int64_t> pos(start.begin(), start.end() - 1);
    for (int64_t e = 0; e < E; ++e) perm[pos[color[e]]++] = (int32_t)e;
  }
  // colour-sorted restriction with first-writer and Dirichlet flags; sorted vertices
  std::vector<uint32_t> emap;
  std::vector<double> svert;
  std::vector<uint8_t> seen;
  try {
    emap.resize(E * nd);
    svert.resize(E * 24);
    seen.assign(nL, 0);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation");
  }
  for (int64_t sidx = 0; sidx < E; ++sidx) {
    const int64_t e = perm[sidx];
    const uint32_t *row = &map[e * nd];
    uint32_t *dst = &emap[sidx * nd];
    for (int64_t n = 0; n < nd; ++n) {
      const uint32_t v = row[n];
      uint32_t f = v;
      if (!seen[v]) {
        f |= FLAG_FIRST;
        seen[v] = 1;
      }
      if (!dir.empty() && dir[v]) f |= FLAG_DIR;
      dst[n] = f;
    }
    std::memcpy(&svert[sidx * 24], &vert[e * 24], 24 * sizeof(double));
  }
  // last writer of every node: scan the sorted order backwards
  std::fill(seen.begin(), seen.end(), 0);
  for (int64_t sidx = E - 1; sidx >= 0; --sidx) {
    uint32_t *dst = &emap[sidx * nd];
    for (int64_t n = 0; n < nd; ++n) {
      const uint32_t v = dst[n] & DOF_MASK;
      if (!seen[v]) {
        dst[n] |= FLAG_LAST;
        seen[v] = 1;
      }
    }
  }

  if (int st = detect_bricks(m.get(), map, perm, dir, s)) return st;
  CEED_CUDA_CHECK(cudaMalloc(&m->d_emap, E * nd * 4));
  CEED_CUDA_CHECK(cudaMalloc(&m->d_perm, E * 4));
  CEED_CUDA_CHECK(cudaMalloc(&m->d_vertices, E * 24 * 8));
  CEED_CUDA_CHECK(cudaMalloc(&m->d_err, sizeof(int) * 4));
  CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_emap, emap.data(), E * nd * 4, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_perm, perm.data(), E * 4, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_vertices, svert.data(), E * 24 * 8, cudaMemcpyHostToDevice, s));
  CEED_CUDA_CHECK(cudaMemsetAsync(m->d_err, 0, sizeof(int) * 4, s));
  if (desc->coords) {  // curved geometry: the handle keeps its own copy of the node positions
    CEED_CUDA_CHECK(cudaMalloc(&m->d_coords, nL * 3 * sizeof(double)));
    CEED_CUDA_CHECK(cudaMemcpyAsync(m->d_coords, desc->coords, nL * 3 * sizeof(double), cudaMemcpyDefault, s));
  }
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  *out = m.release();
  return CEED_OK;
}

extern "C" int ceed_destroy_mesh(ceed_mesh_t m) {
  if (!m) return CEED_OK;
  cudaDeviceSynchronize();
  HostFree()(m);
  return CEED_OK;
}

extern "C" int ceed_mesh_info(ceed_mesh_t m, int32_t *n_colors, int32_t *Q, int32_t *P) {
  if (int st = check_mesh(m)) return st;
  if (n_colors) *n_colors = m->n_colors;
  if (Q) *Q = m->Q;
  if (P) *P = m->P;
  return CEED_OK;
}

extern "C" int ceed_mesh_bricks(ceed_mesh_t m, int64_t *n_bricks) {
  if (int st = check_mesh(m)) return st;
  if (!n_bricks) return fail(CEED_ERR_INVALID, "null output");
  *n_bricks = m->n_bricks;
  return CEED_OK;
}

extern "C" int ceed_set_wait_limits(int64_t copy_polls, int64_t barrier_polls) {
  if (copy_polls > 0 || barrier_polls > WAIT_GRID_DEFAULT)
    return fail(CEED_ERR_INVALID, "copy_polls must be negative (default) or 0; barrier_polls at most the default");
  g_copy_wait.store(copy_polls < 0 ? WAIT_COPY_DEFAULT : (int)copy_polls, std::memory_order_relaxed);
  g_grid_wait.store(barrier_polls < 0 ? WAIT_GRID_DEFAULT : (long long)barrier_polls, std::memory_order_relaxed);
  return CEED_OK;
}

extern "C" int ceed_mesh_status(ceed_mesh_t m, void *stream) {
  if (int st = check_mesh(m)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  CEED_CUDA_CHECK(cudaMemcpyAsync(&err, m->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  if (err) {
    CEED_CUDA_CHECK(cudaMemsetAsync(m->d_err + 1, 0, sizeof(int), s));
    CEED_CUDA_CHECK(cudaStreamSynchronize(s));
    return fail(CEED_ERR_TIMEOUT, "an apply kernel's quadrature-data copy wait gave up");
  }
  return CEED_OK;
}

size_t ceedgb::prec_size(int prec) {
  switch (prec) {
    case CEED_F64:
    case CEED_F64_DF: return 8;
    case CEED_F32:
    case CEED_F32_GEO: return 4;
    case CEED_BF16:
    case CEED_F16: return 2;
    default: return 0;
  }
}

extern "C" size_t ceed_qdata_bytes(ceed_mesh_t m, int op, int prec) {
  if (!m || prec_size(prec) == 0 || (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION)) return 0;
  if (prec == CEED_F32_GEO) {
    if (op != CEED_OP_DIFFUSION) return 0;
    op = OP_DIFF_GEO;
  }
  return (size_t)m->E * qdata_estride(op, prec_size(prec), m->Q) * prec_size(prec);
}

static int apply_common(ceed_mesh_t m, int op, const void *qdata, int prec, const double *x, double *y, int nrhs,
                        unsigned flags, void *stream) {
  if (int st = check_mesh(m)) return st;
  if (!qdata || !x || !y) return fail(CEED_ERR_INVALID, "null qdata, x or y");
  if (x == y) return fail(CEED_ERR_INVALID, "x and y must not alias");
  if (nrhs < 1) return fail(CEED_ERR_INVALID, "nrhs must be >= 1");
  if (prec_size(prec) == 0) return fail(CEED_ERR_INVALID, "unknown precision");
  if (prec < CEED_F64 || prec > CEED_F64_DF) return fail(CEED_ERR_INVALID, "unknown precision");
  ApplyReq r;
  r.op = op;
  r.prec = prec;
  r.qdata = qdata;
  r.x = x;
  r.y = y;
  r.ncol = m->ncomp * nrhs;
  r.masked = (flags & CEED_APPLY_DIRICHLET) ? 1 : 0;
  if (r.masked && !m->has_dirichlet) return fail(CEED_ERR_INVALID, "mesh has no Dirichlet mask");
  return launch_apply(m, r, (cudaStream_t)stream);
}

extern "C" int ceed_apply_mass(ceed_mesh_t m, const void *qdata, int prec, const double *x, double *y, int nrhs,
                               unsigned flags, void *stream) {
  return apply_common(m, CEED_OP_MASS, qdata, prec, x, y, nrhs, flags, stream);
}

extern "C" int ceed_apply_diffusion(ceed_mesh_t m, const void *qdata, int prec, const double *x, double *y, int nrhs,
                                    unsigned flags, void *stream) {
  return apply_common(m, CEED_OP_DIFFUSION, qdata, prec, x, y, nrhs, flags, stream);
}

extern "C" int ceed_apply_host(ceed_mesh_t m, int op, const void *qdata, int prec, const double *x_host,
                               double *y_host, double *x_dev, double *y_dev, int nrhs, unsigned flags, void *stream) {
  if (int st = check_mesh(m)) return st;
  if (!x_host || !y_host || !x_dev || !y_dev) return fail(CEED_ERR_INVALID, "null host or device buffer");
  if (x_dev == y_dev) return fail(CEED_ERR_INVALID, "x_dev and y_dev must not alias");
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  if (nrhs < 1) return fail(CEED_ERR_INVALID, "nrhs must be >= 1");
  const size_t bytes = (size_t)m->n_ldof * (size_t)m->ncomp * (size_t)nrhs * sizeof(double);
  cudaStream_t s = (cudaStream_t)stream;
  CEED_CUDA_CHECK(cudaMemcpyAsync(x_dev, x_host, bytes, cudaMemcpyHostToDevice, s));
  if (int st = apply_common(m, op, qdata, prec, x_dev, y_dev, nrhs, flags, stream)) return st;
  CEED_CUDA_CHECK(cudaMemcpyAsync(y_host, y_dev, bytes, cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  return CEED_OK;
}

// The brick kernel serves FP32-pipe operators (FP32 arithmetic on FP32, BF16, FP16 or on-the-fly
// geometry data) with one column, on meshes whose setup found a brick lattice.
static bool brick_ok(ceed_mesh_t m, int prec, int ncol) {
  return m->n_bricks > 0 && ncol == 1 &&
         (prec == CEED_F32 || prec == CEED_BF16 || prec == CEED_F16 || prec == CEED_F32_GEO);
}

// ---------------------------------------------------------------------------------------------
// Autotuner for the apply kernel: times every (elements per block, staging) variant on the
// caller's mesh, quadrature data and vectors, and keeps the fastest for (op, prec) in the handle.
extern "C" int ceed_autotune_apply(ceed_mesh_t m, int op, const void *qdata, int prec, const double *x, double *y,
                                   int nrhs, int32_t *best_ne, int32_t *best_stage, float *best_ms, void *stream) {
  if (int st = check_mesh(m)) return st;
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  if (prec < CEED_F64 || prec > CEED_F64_DF) return fail(CEED_ERR_INVALID, "unknown precision");
  if (!qdata || !x || !y || x == y || nrhs < 1) return fail(CEED_ERR_INVALID, "bad autotune arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int ne_max = std::min(32, std::max(1, 256 / (m->Q * m->Q)));
  ApplyReq r;
  r.op = op;
  r.prec = prec;
  r.qdata = qdata;
  r.x = x;
  r.y = y;
  r.ncol = m->ncomp * nrhs;
  r.masked = 0;
  cudaEvent_t e0, e1;
  CEED_CUDA_CHECK(cudaEventCreate(&e0));
  CEED_CUDA_CHECK(cudaEventCreate(&e1));
  ApplyChoice best;
  best.ms = 1e30f;
  const int reps = 3;
  const bool bricks = brick_ok(m, prec, r.ncol);
  for (int stage = 0; stage <= (bricks ? 3 : 1); ++stage) {
    for (int ne = 1; ne <= (stage >= 2 ? 1 : ne_max); ne *= 2) {  // the brick kernel has one shape
      r.ne = ne;
      r.stage = stage;
      if (launch_apply(m, r, s) != CEED_OK) continue;  // e.g. shared memory beyond the limit
      cudaEventRecord(e0, s);
      for (int k = 0; k < reps; ++k) launch_apply(m, r, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (ms < best.ms) {
        best.ms = ms;
        best.ne = ne;
        best.stage = stage;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CEED_CUDA_CHECK(cudaGetLastError());
  if (best.ne == 0) return fail(CEED_ERR_CUDA, "no apply variant ran");
  m->tuned[op][prec] = best;
  if (best_ne) *best_ne = best.ne;
  if (best_stage) *best_stage = best.stage;
  if (best_ms) *best_ms = best.ms;
  return CEED_OK;
}

extern "C" int ceed_set_apply_variant(ceed_mesh_t m, int op, int prec, int ne, int stage) {
  if (int st = check_mesh(m)) return st;
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "unknown operator");
  if (prec < CEED_F64 || prec > CEED_F64_DF) return fail(CEED_ERR_INVALID, "unknown precision");
  if (ne < 0 || ne > std::min(32, std::max(1, 256 / (m->Q * m->Q))) || stage < 0 || stage > 3)
    return fail(CEED_ERR_INVALID, "elements per block must be 0 (default) .. min(32, 256 / Q^2), stage 0 .. 3");
  if (stage >= 2 && !brick_ok(m, prec, 1))
    return fail(CEED_ERR_INVALID, "stage 2 and 3 (brick kernel) need a brick lattice and an FP32-pipe precision");
  if (stage >= 2 && ne == 0) ne = 1;  // the brick kernel has one shape (ne = 0 would restore the default)
  m->tuned[op][prec].ne = ne;
  m->tuned[op][prec].stage = stage;
  m->tuned[op][prec].ms = 0.f;
  return CEED_OK;
}
