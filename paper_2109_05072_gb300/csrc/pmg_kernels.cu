// p-multigrid transfers between two orders on the same elements.
//
// Prolongation u_f = P u_c evaluates the coarse element polynomial at the fine GLL nodes with the
// 1D interpolation matrix B (P_f x P_c) applied along r, s, t (sum factorization).  A continuous
// coarse function gives the same value at a shared fine node from every element, so the first
// element (in colour order) that holds the node writes it: one launch, no conflicts.
// Restriction r_c = P^T r_f is the exact transpose of that assembled P: each fine node enters once
// (through its first-writer element), B^T is applied along t, s, r, and the coarse element vectors
// are scatter-added colour by colour (atomic-free, deterministic).
// Dirichlet nodes carry zero in both directions (the corrections live in the constrained space).
#include "internal.h"

namespace ceedgb {

struct TransferArgs {
  const uint32_t *emap_c, *emap_f;
  const double *in;
  double *out;
  int64_t e_begin, e_count;
  int Pc, Pf;
  int add;                       // prolongation: out += P in (1) or out = P in (0)
  double B[MAX_P * MAX_P];       // B[i * Pc + a] = coarse basis a at fine node i
};

constexpr int TR_THREADS = 128;

__global__ void __launch_bounds__(TR_THREADS) prolong_kernel(const TransferArgs t) {
  const int64_t e = t.e_begin + blockIdx.x;
  if (e >= t.e_begin + t.e_count) return;
  __shared__ double uc[MAX_P * MAX_P * MAX_P];
  __shared__ double t1[MAX_P * MAX_P * MAX_P];
  __shared__ double t2[MAX_P * MAX_P * MAX_P];
  const int Pc = t.Pc, Pf = t.Pf;
  const int ncn = Pc * Pc * Pc, nfn = Pf * Pf * Pf;
  for (int n = threadIdx.x; n < ncn; n += blockDim.x) {
    const uint32_t v = t.emap_c[e * ncn + n];
    uc[n] = (v & FLAG_DIR) ? 0.0 : t.in[v & DOF_MASK];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Pc * Pc * Pf; o += blockDim.x) {  // r: (c, b, i)
    const int i = o % Pf, b = (o / Pf) % Pc, c = o / (Pf * Pc);
    double s = 0.0;
    for (int a = 0; a < Pc; ++a) s += t.B[i * Pc + a] * uc[(c * Pc + b) * Pc + a];
    t1[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Pc * Pf * Pf; o += blockDim.x) {  // s: (c, j, i)
    const int i = o % Pf, j = (o / Pf) % Pf, c = o / (Pf * Pf);
    double s = 0.0;
    for (int b = 0; b < Pc; ++b) s += t.B[j * Pc + b] * t1[(c * Pc + b) * Pf + i];
    t2[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nfn; o += blockDim.x) {  // t: (k, j, i), written by the node's first writer
    const uint32_t v = t.emap_f[e * nfn + o];
    if (!(v & FLAG_FIRST)) continue;
    const int i = o % Pf, j = (o / Pf) % Pf, k = o / (Pf * Pf);
    double s = 0.0;
    for (int c = 0; c < Pc; ++c) s += t.B[k * Pc + c] * t2[(c * Pf + j) * Pf + i];
    if (v & FLAG_DIR) s = 0.0;
    const int64_t dof = v & DOF_MASK;
    t.out[dof] = t.add ? t.out[dof] + s : s;
  }
}

__global__ void __launch_bounds__(TR_THREADS) restrict_kernel(const TransferArgs t) {
  const int64_t e = t.e_begin + blockIdx.x;
  if (e >= t.e_begin + t.e_count) return;
  __shared__ double rf[MAX_P * MAX_P * MAX_P];
  __shared__ double t2[MAX_P * MAX_P * MAX_P];
  __shared__ double t1[MAX_P * MAX_P * MAX_P];
  const int Pc = t.Pc, Pf = t.Pf;
  const int ncn = Pc * Pc * Pc, nfn = Pf * Pf * Pf;
  for (int n = threadIdx.x; n < nfn; n += blockDim.x) {
    const uint32_t v = t.emap_f[e * nfn + n];
    rf[n] = ((v & FLAG_FIRST) && !(v & FLAG_DIR)) ? t.in[v & DOF_MASK] : 0.0;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Pc * Pf * Pf; o += blockDim.x) {  // t^T: (c, j, i)
    const int i = o % Pf, j = (o / Pf) % Pf, c = o / (Pf * Pf);
    double s = 0.0;
    for (int k = 0; k < Pf; ++k) s += t.B[k * Pc + c] * rf[(k * Pf + j) * Pf + i];
    t2[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Pc * Pc * Pf; o += blockDim.x) {  // s^T: (c, b, i)
    const int i = o % Pf, b = (o / Pf) % Pc, c = o / (Pf * Pc);
    double s = 0.0;
    for (int j = 0; j < Pf; ++j) s += t.B[j * Pc + b] * t2[(c * Pf + j) * Pf + i];
    t1[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ncn; o += blockDim.x) {  // r^T: (c, b, a), scatter-add to the coarse vector
    const int a = o % Pc, b = (o / Pc) % Pc, c = o / (Pc * Pc);
    double s = 0.0;
    for (int i = 0; i < Pf; ++i) s += t.B[i * Pc + a] * t1[(c * Pc + b) * Pf + i];
    const uint32_t v = t.emap_c[e * ncn + o];
    const int64_t dof = v & DOF_MASK;
    if (v & FLAG_DIR) {
      if (v & FLAG_FIRST) t.out[dof] = 0.0;
    } else if (v & FLAG_FIRST) {
      t.out[dof] = s;
    } else {
      t.out[dof] += s;
    }
  }
}

static void transfer_table(ceed_mesh_t coarse, ceed_mesh_t fine, double *B) {
  // coarse GLL Lagrange basis at the fine GLL nodes, barycentric form
  const int Pc = coarse->P, Pf = fine->P;
  const double *xc = coarse->gll_x, *xf = fine->gll_x;
  double lam[MAX_P];
  for (int a = 0; a < Pc; ++a) {
    double d = 1.0;
    for (int m = 0; m < Pc; ++m)
      if (m != a) d *= xc[a] - xc[m];
    lam[a] = 1.0 / d;
  }
  for (int i = 0; i < Pf; ++i) {
    int hit = -1;
    for (int a = 0; a < Pc; ++a)
      if (xf[i] == xc[a]) hit = a;
    double den = 0.0;
    if (hit < 0)
      for (int a = 0; a < Pc; ++a) den += lam[a] / (xf[i] - xc[a]);
    for (int a = 0; a < Pc; ++a)
      B[i * Pc + a] = (hit >= 0) ? (a == hit ? 1.0 : 0.0) : (lam[a] / (xf[i] - xc[a])) / den;
  }
}

int check_transfer_pair(ceed_mesh_t coarse, ceed_mesh_t fine) {
  if (!coarse || !fine) return fail(CEED_ERR_INVALID, "null mesh in a transfer");
  if (coarse->E != fine->E) return fail(CEED_ERR_INVALID, "p-multigrid levels must share the elements");
  if (coarse->P >= fine->P) return fail(CEED_ERR_INVALID, "coarse level must have a lower order");
  if (coarse->n_colors != fine->n_colors) return fail(CEED_ERR_INVALID, "levels are coloured differently");
  for (int c = 0; c <= fine->n_colors; ++c)
    if (coarse->color_start[c] != fine->color_start[c]) return fail(CEED_ERR_INVALID, "levels are coloured differently");
  if (coarse->ncomp != 1 || fine->ncomp != 1) return fail(CEED_ERR_UNSUPPORTED, "p-multigrid needs ncomp = 1");
  return CEED_OK;
}

int launch_prolong(ceed_mesh_t coarse, ceed_mesh_t fine, const double *uc, double *uf, int add, cudaStream_t s) {
  TransferArgs t;
  t.emap_c = coarse->d_emap;
  t.emap_f = fine->d_emap;
  t.in = uc;
  t.out = uf;
  t.Pc = coarse->P;
  t.Pf = fine->P;
  t.add = add;
  transfer_table(coarse, fine, t.B);
  t.e_begin = 0;
  t.e_count = fine->E;
  prolong_kernel<<<(unsigned)fine->E, TR_THREADS, 0, s>>>(t);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

int launch_restrict(ceed_mesh_t coarse, ceed_mesh_t fine, const double *rf, double *rc, cudaStream_t s) {
  TransferArgs t;
  t.emap_c = coarse->d_emap;
  t.emap_f = fine->d_emap;
  t.in = rf;
  t.out = rc;
  t.Pc = coarse->P;
  t.Pf = fine->P;
  t.add = 0;
  transfer_table(coarse, fine, t.B);
  for (int c = 0; c < coarse->n_colors; ++c) {
    t.e_begin = coarse->color_start[c];
    t.e_count = coarse->color_start[c + 1] - t.e_begin;
    if (t.e_count == 0) continue;
    restrict_kernel<<<(unsigned)t.e_count, TR_THREADS, 0, s>>>(t);
  }
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

}  // namespace ceedgb
