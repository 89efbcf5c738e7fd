// Conforming hp (variable order) operator on a structured hexahedral lattice: the mixed-order
// elements of the batched workload joined into one continuous space (minimum rule: every face and
// edge carries the lowest order of the elements sharing it).
//
// The space is the image of a conforming prolongation P from true dofs to element nodes.  Vertices
// carry one value; an edge of order p carries its interior GLL(p) nodes, and its polynomial is the
// 1D Lagrange interpolant through those and its two vertices; a face of order p carries its
// interior GLL(p)^2 nodes and equals its edges' polynomials on its boundary; an element carries its
// interior nodes.  An element node takes the value of the polynomial of the lowest-dimensional
// entity it lies on, so a row of P is either one true dof (the node is that dof) or the Lagrange
// weights of a lower-order entity, composed through lower-order edges.  The operator on true dofs
// is y = P^T blockdiag(A_e) P x: P x gathers element vectors, the fused tensor-product kernels apply
// every order group (each group a mesh whose nodes are its element vectors, one colour), and P^T
// sums back in a fixed order (a CSR of P^T, deterministic).
//
// True-dof numbering (documented in the header): vertices (i fastest); edges along x, y, z, each
// axis by lower vertex with i fastest, interior nodes in increasing coordinate; faces normal to x,
// y, z, by lower corner, interior nodes with the first in-plane axis fastest; element interiors in
// element order, a fastest.  Element-node rows of P are ordered by order group (ascending order),
// element (ascending index), node (a fastest).
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

struct ceed_hp_s {
  int device = 0;
  int nx = 0, ny = 0, nz = 0;
  int64_t E = 0, n_true = 0, n_rows = 0;
  int q_rule = 0;
  bool dirichlet = false;
  struct Group {
    int p = 0;
    int64_t n_elem = 0, row0 = 0;     // element count, first E-vector row
    ceed_mesh_t mesh = nullptr;       // identity restriction over the group's element vectors
    void *qdata[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // [op][prec: F64, F32, F64_DF]
  };
  std::vector<Group> groups;
  int64_t *d_prow = nullptr;     // CSR of P: [n_rows + 1]
  int64_t *d_pcol = nullptr;     // true-dof column indices
  double *d_pval = nullptr;
  int64_t *d_trow = nullptr;     // CSR of P^T: [n_true + 1]
  int64_t *d_tcol = nullptr;     // E-vector rows
  double *d_tval = nullptr;
  uint8_t *d_dir = nullptr;      // [n_true] Dirichlet flags
  double *d_u = nullptr, *d_v = nullptr;   // element-vector work arrays [n_rows]
};

namespace ceedgb {
namespace {

// Lagrange weights of the nodes x[0..n) at t, product formula (exactly 1 and 0 at a node).
void lagrange_weights(int n, const double *x, double t, double *w) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= (t - x[m]) / (x[j] - x[m]);
    w[j] = v;
  }
}

struct Row {
  std::vector<std::pair<int64_t, double>> t;
  void add(int64_t q, double w) { t.emplace_back(q, w); }
  void finish() {
    std::sort(t.begin(), t.end());
    std::vector<std::pair<int64_t, double>> o;
    for (auto &e : t) {
      if (!o.empty() && o.back().first == e.first) o.back().second += e.second;
      else o.push_back(e);
    }
    t.swap(o);
  }
};

struct Builder {
  int n[3];
  const std::vector<int> &ord;
  std::vector<int> eord[3], ford[3];
  std::vector<int64_t> ebase[3], fbase[3], cbase;
  std::vector<double> gx[MAX_P + 1];   // GLL nodes of each order
  int64_t nT = 0;

  explicit Builder(int nx, int ny, int nz, const std::vector<int> &o) : ord(o) {
    n[0] = nx;
    n[1] = ny;
    n[2] = nz;
    for (int p = 1; p < MAX_P; ++p) {
      double w[MAX_P];
      gx[p].resize(p + 1);
      gll_rule(p + 1, gx[p].data(), w);
    }
  }
  int elem_order(int ex, int ey, int ez) const { return ord[ex + (int64_t)n[0] * (ey + (int64_t)n[1] * ez)]; }
  void eext(int d, int64_t e[3]) const {
    for (int a = 0; a < 3; ++a) e[a] = n[a] + 1;
    e[d] -= 1;
  }
  void fext(int d, int64_t f[3]) const {
    for (int a = 0; a < 3; ++a) f[a] = n[a];
    f[d] += 1;
  }
  int64_t eidx(int d, int i, int j, int k) const {
    int64_t e[3];
    eext(d, e);
    return i + e[0] * (j + e[1] * (int64_t)k);
  }
  int64_t fidx(int d, int i, int j, int k) const {
    int64_t f[3];
    fext(d, f);
    return i + f[0] * (j + f[1] * (int64_t)k);
  }
  int64_t vdof(int i, int j, int k) const { return i + (n[0] + 1) * (j + (int64_t)(n[1] + 1) * k); }

  void orders_and_numbering() {
    const int big = 1 << 30;
    for (int d = 0; d < 3; ++d) {
      int64_t e[3], f[3];
      eext(d, e);
      fext(d, f);
      eord[d].assign(e[0] * e[1] * e[2], big);
      ford[d].assign(f[0] * f[1] * f[2], big);
    }
    // every element lowers the order of its 12 edges and 6 faces
    for (int ez = 0; ez < n[2]; ++ez)
      for (int ey = 0; ey < n[1]; ++ey)
        for (int ex = 0; ex < n[0]; ++ex) {
          const int p = elem_order(ex, ey, ez);
          const int c[3] = {ex, ey, ez};
          for (int d = 0; d < 3; ++d) {
            const int o0 = (d + 1) % 3, o1 = (d + 2) % 3;
            for (int s0 = 0; s0 < 2; ++s0)
              for (int s1 = 0; s1 < 2; ++s1) {
                int v[3] = {c[0], c[1], c[2]};
                v[o0] += s0;
                v[o1] += s1;
                int &eo = eord[d][eidx(d, v[0], v[1], v[2])];
                eo = std::min(eo, p);
              }
            for (int s = 0; s < 2; ++s) {
              int v[3] = {c[0], c[1], c[2]};
              v[d] += s;
              int &fo = ford[d][fidx(d, v[0], v[1], v[2])];
              fo = std::min(fo, p);
            }
          }
        }
    nT = (int64_t)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
    for (int d = 0; d < 3; ++d) {
      ebase[d].resize(eord[d].size());
      for (size_t i = 0; i < eord[d].size(); ++i) {
        ebase[d][i] = nT;
        nT += eord[d][i] - 1;
      }
    }
    for (int d = 0; d < 3; ++d) {
      fbase[d].resize(ford[d].size());
      for (size_t i = 0; i < ford[d].size(); ++i) {
        fbase[d][i] = nT;
        nT += (int64_t)(ford[d][i] - 1) * (ford[d][i] - 1);
      }
    }
    cbase.resize(ord.size());
    for (size_t e = 0; e < ord.size(); ++e) {
      cbase[e] = nT;
      nT += (int64_t)(ord[e] - 1) * (ord[e] - 1) * (ord[e] - 1);
    }
  }

  // the edge polynomial along axis d with lower vertex v, at reference coordinate t
  void edge_value(int d, const int v[3], double t, double scale, Row &r) const {
    const int64_t ei = eidx(d, v[0], v[1], v[2]);
    const int p = eord[d][ei];
    double w[MAX_P + 1];
    lagrange_weights(p + 1, gx[p].data(), t, w);
    for (int m = 0; m <= p; ++m) {
      if (w[m] == 0.0) continue;
      if (m == 0) {
        r.add(vdof(v[0], v[1], v[2]), scale * w[m]);
      } else if (m == p) {
        int u[3] = {v[0], v[1], v[2]};
        u[d] += 1;
        r.add(vdof(u[0], u[1], u[2]), scale * w[m]);
      } else {
        r.add(ebase[d][ei] + (m - 1), scale * w[m]);
      }
    }
  }

  // the face polynomial normal to axis d with lower corner v, at in-plane coordinates (s, t)
  // along the lower and the higher of the two other axes
  void face_value(int d, const int v[3], double s, double t, double scale, Row &r) const {
    const int o0 = d == 0 ? 1 : 0, o1 = d == 2 ? 1 : 2;
    const int64_t fi = fidx(d, v[0], v[1], v[2]);
    const int p = ford[d][fi];
    double ws[MAX_P + 1], wt[MAX_P + 1];
    lagrange_weights(p + 1, gx[p].data(), s, ws);
    lagrange_weights(p + 1, gx[p].data(), t, wt);
    for (int m1 = 0; m1 <= p; ++m1) {
      if (ws[m1] == 0.0) continue;
      for (int m2 = 0; m2 <= p; ++m2) {
        if (wt[m2] == 0.0) continue;
        const double w = scale * ws[m1] * wt[m2];
        const bool b1 = m1 == 0 || m1 == p, b2 = m2 == 0 || m2 == p;
        int c[3] = {v[0], v[1], v[2]};
        if (b1 && b2) {
          c[o0] += m1 == p;
          c[o1] += m2 == p;
          r.add(vdof(c[0], c[1], c[2]), w);
        } else if (b1) {
          c[o0] += m1 == p;
          edge_value(o1, c, gx[p][m2], w, r);
        } else if (b2) {
          c[o1] += m2 == p;
          edge_value(o0, c, gx[p][m1], w, r);
        } else {
          r.add(fbase[d][fi] + (m1 - 1) + (int64_t)(p - 1) * (m2 - 1), w);
        }
      }
    }
  }

  // row of P for node (a, b, c) of element e
  void node_row(int64_t e, int a, int b, int c, Row &r) const {
    const int ex = (int)(e % n[0]), ey = (int)((e / n[0]) % n[1]), ez = (int)(e / ((int64_t)n[0] * n[1]));
    const int p = ord[e];
    const int idx[3] = {a, b, c};
    const int base[3] = {ex, ey, ez};
    bool bnd[3];
    int nb = 0;
    for (int d = 0; d < 3; ++d) {
      bnd[d] = idx[d] == 0 || idx[d] == p;
      nb += bnd[d];
    }
    int v[3];
    for (int d = 0; d < 3; ++d) v[d] = base[d] + ((bnd[d] && idx[d] == p) ? 1 : 0);
    if (nb == 3) {
      r.add(vdof(v[0], v[1], v[2]), 1.0);
    } else if (nb == 2) {
      const int d = !bnd[0] ? 0 : !bnd[1] ? 1 : 2;
      edge_value(d, v, gx[p][idx[d]], 1.0, r);
    } else if (nb == 1) {
      const int d = bnd[0] ? 0 : bnd[1] ? 1 : 2;
      const int o0 = d == 0 ? 1 : 0, o1 = d == 2 ? 1 : 2;
      face_value(d, v, gx[p][idx[o0]], gx[p][idx[o1]], 1.0, r);
    } else {
      const int P = p - 1;
      r.add(cbase[e] + (a - 1) + (int64_t)P * ((b - 1) + (int64_t)P * (c - 1)), 1.0);
    }
    r.finish();
  }

  // Dirichlet flags of the true dofs on the lattice boundary
  void boundary(std::vector<uint8_t> &dir) const {
    dir.assign(nT, 0);
    for (int k = 0; k <= n[2]; ++k)
      for (int j = 0; j <= n[1]; ++j)
        for (int i = 0; i <= n[0]; ++i)
          if (i == 0 || i == n[0] || j == 0 || j == n[1] || k == 0 || k == n[2]) dir[vdof(i, j, k)] = 1;
    for (int d = 0; d < 3; ++d) {
      int64_t e[3], f[3];
      eext(d, e);
      fext(d, f);
      for (int64_t k = 0; k < e[2]; ++k)
        for (int64_t j = 0; j < e[1]; ++j)
          for (int64_t i = 0; i < e[0]; ++i) {
            const int64_t v[3] = {i, j, k};
            bool on = false;
            for (int a = 0; a < 3; ++a)
              if (a != d && (v[a] == 0 || v[a] == n[a])) on = true;
            if (!on) continue;
            const int64_t ei = i + e[0] * (j + e[1] * k);
            for (int m = 1; m < eord[d][ei]; ++m) dir[ebase[d][ei] + m - 1] = 1;
          }
      for (int64_t k = 0; k < f[2]; ++k)
        for (int64_t j = 0; j < f[1]; ++j)
          for (int64_t i = 0; i < f[0]; ++i) {
            const int64_t v[3] = {i, j, k};
            if (v[d] != 0 && v[d] != n[d]) continue;
            const int64_t fi = i + f[0] * (j + f[1] * k);
            const int64_t cnt = (int64_t)(ford[d][fi] - 1) * (ford[d][fi] - 1);
            for (int64_t m = 0; m < cnt; ++m) dir[fbase[d][fi] + m] = 1;
          }
    }
  }
};

// y[r] = sum_k val[k] x[col[k]] over row r's entries; masked: columns flagged Dirichlet read 0.
__global__ void hp_spmv_kernel(int64_t rows, const int64_t *__restrict__ rp, const int64_t *__restrict__ col,
                               const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
                               const uint8_t *__restrict__ dir, int masked) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double acc = 0.0;
  for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
    const int64_t c = col[k];
    if (masked && dir[c]) continue;
    acc += val[k] * x[c];
  }
  y[r] = acc;
}

// y = P^T v in the fixed order of the CSR of P^T; masked: y = x on Dirichlet dofs.
__global__ void hp_spmv_t_kernel(int64_t rows, const int64_t *__restrict__ rp, const int64_t *__restrict__ col,
                                 const double *__restrict__ val, const double *__restrict__ v,
                                 const double *__restrict__ x, double *__restrict__ y,
                                 const uint8_t *__restrict__ dir, int masked) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  if (masked && dir[r]) {
    y[r] = x[r];
    return;
  }
  double acc = 0.0;
  for (int64_t k = rp[r]; k < rp[r + 1]; ++k) acc += val[k] * v[col[k]];
  y[r] = acc;
}

struct HpFree {
  void operator()(ceed_hp_s *h) const {
    if (!h) return;
    for (auto &g : h->groups) {
      if (g.mesh) ceed_destroy_mesh(g.mesh);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) cudaFree(g.qdata[a][b]);
    }
    cudaFree(h->d_prow);
    cudaFree(h->d_pcol);
    cudaFree(h->d_pval);
    cudaFree(h->d_trow);
    cudaFree(h->d_tcol);
    cudaFree(h->d_tval);
    cudaFree(h->d_dir);
    cudaFree(h->d_u);
    cudaFree(h->d_v);
    delete h;
  }
};

template <typename T>
int upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
  CEED_CUDA_CHECK(cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(T)));
  if (!src.empty()) CEED_CUDA_CHECK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return CEED_OK;
}

// The host part of the space: true-dof count, order groups (ascending order, element lists) and
// the CSR of P with rows in group order, plus the Dirichlet flag of every true dof.
struct HostP {
  int64_t n_true = 0, rows = 0;
  std::vector<int> porders;
  std::vector<std::vector<int64_t>> members;
  std::vector<int64_t> prow, pcol;
  std::vector<double> pval;
  std::vector<uint8_t> dir;
};

int build_host_p(int nx, int ny, int nz, const std::vector<int> &ord, HostP &H) {
  const int64_t E = (int64_t)nx * ny * nz;
  try {
    Builder B(nx, ny, nz, ord);
    B.orders_and_numbering();
    H.n_true = B.nT;
    if (B.nT >= ((int64_t)1 << 40)) return fail(CEED_ERR_INVALID, "mesh too large");
    H.porders.assign(ord.begin(), ord.end());
    std::sort(H.porders.begin(), H.porders.end());
    H.porders.erase(std::unique(H.porders.begin(), H.porders.end()), H.porders.end());
    H.members.assign(H.porders.size(), {});
    for (int64_t e = 0; e < E; ++e)
      H.members[std::lower_bound(H.porders.begin(), H.porders.end(), ord[e]) - H.porders.begin()].push_back(e);
    H.rows = 0;
    for (size_t g = 0; g < H.porders.size(); ++g)
      H.rows += (int64_t)H.members[g].size() * (H.porders[g] + 1) * (H.porders[g] + 1) * (H.porders[g] + 1);
    H.prow.assign(H.rows + 1, 0);
    H.pcol.clear();
    H.pval.clear();
    H.pcol.reserve(H.rows + H.rows / 2);
    H.pval.reserve(H.rows + H.rows / 2);
    Row r;
    int64_t ri = 0;
    for (size_t g = 0; g < H.porders.size(); ++g) {
      const int P = H.porders[g] + 1;
      for (int64_t e : H.members[g])
        for (int c = 0; c < P; ++c)
          for (int b = 0; b < P; ++b)
            for (int a = 0; a < P; ++a) {
              r.t.clear();
              B.node_row(e, a, b, c, r);
              for (auto &kv : r.t) {
                H.pcol.push_back(kv.first);
                H.pval.push_back(kv.second);
              }
              H.prow[++ri] = (int64_t)H.pcol.size();
            }
    }
    B.boundary(H.dir);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation while building the conforming prolongation");
  }
  return CEED_OK;
}

int check_orders(int nx, int ny, int nz, const int32_t *orders, std::vector<int> &ord) {
  if (nx < 1 || ny < 1 || nz < 1) return fail(CEED_ERR_INVALID, "nx, ny, nz must be >= 1");
  if (!orders) return fail(CEED_ERR_INVALID, "orders (host) are required");
  const int64_t E = (int64_t)nx * ny * nz;
  ord.resize(E);
  for (int64_t e = 0; e < E; ++e) {
    ord[e] = orders[e];
    if (ord[e] < 1 || ord[e] > 8) return fail(CEED_ERR_INVALID, "orders must be in 1..8");
  }
  return CEED_OK;
}

}  // namespace
}  // namespace ceedgb

using namespace ceedgb;

extern "C" int ceed_hp_prolongation(int32_t nx, int32_t ny, int32_t nz, const int32_t *orders, int64_t *n_true,
                                    int64_t *n_rows, int64_t *nnz, int64_t *row_ptr, int64_t *col, double *val,
                                    uint8_t *dirichlet) {
  if (!n_true || !n_rows || !nnz) return fail(CEED_ERR_INVALID, "null size output");
  const bool fill = row_ptr || col || val || dirichlet;
  if (fill && !(row_ptr && col && val && dirichlet)) return fail(CEED_ERR_INVALID, "give all four arrays or none");
  std::vector<int> ord;
  if (int st = check_orders(nx, ny, nz, orders, ord)) return st;
  HostP H;
  if (int st = build_host_p(nx, ny, nz, ord, H)) return st;
  *n_true = H.n_true;
  *n_rows = H.rows;
  *nnz = (int64_t)H.pcol.size();
  if (fill) {
    std::memcpy(row_ptr, H.prow.data(), H.prow.size() * sizeof(int64_t));
    std::memcpy(col, H.pcol.data(), H.pcol.size() * sizeof(int64_t));
    std::memcpy(val, H.pval.data(), H.pval.size() * sizeof(double));
    std::memcpy(dirichlet, H.dir.data(), H.dir.size() * sizeof(uint8_t));
  }
  return CEED_OK;
}

extern "C" int ceed_hp_setup(const ceed_hp_desc *desc, ceed_hp_t *out, void *stream) {
  if (!desc || !out) return fail(CEED_ERR_INVALID, "null descriptor or output");
  *out = nullptr;
  if (!desc->vertices) return fail(CEED_ERR_INVALID, "vertices (device) are required");
  if (desc->q_rule != CEED_QRULE_GLL && desc->q_rule != CEED_QRULE_GAUSS) return fail(CEED_ERR_INVALID, "unknown rule");
  std::vector<int> ord;
  if (int st = check_orders(desc->nx, desc->ny, desc->nz, desc->orders, ord)) return st;
  const int64_t E = (int64_t)desc->nx * desc->ny * desc->nz;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<ceed_hp_s, HpFree> h(new (std::nothrow) ceed_hp_s());
  if (!h) return fail(CEED_ERR_OOM, "host allocation");
  CEED_CUDA_CHECK(cudaGetDevice(&h->device));
  h->nx = desc->nx;
  h->ny = desc->ny;
  h->nz = desc->nz;
  h->E = E;
  h->q_rule = desc->q_rule;
  h->dirichlet = desc->dirichlet != 0;

  // P (CSR, rows in group order), the order groups and the Dirichlet flags, built on the host
  HostP H;
  if (int st = build_host_p(desc->nx, desc->ny, desc->nz, ord, H)) return st;
  h->n_true = H.n_true;
  int64_t rows = 0;
  for (size_t g = 0; g < H.porders.size(); ++g) {
    ceed_hp_s::Group G;
    G.p = H.porders[g];
    G.n_elem = (int64_t)H.members[g].size();
    G.row0 = rows;
    rows += G.n_elem * (G.p + 1) * (G.p + 1) * (G.p + 1);
    h->groups.push_back(G);
  }
  h->n_rows = rows;
  const std::vector<int> &porders = H.porders;
  const std::vector<std::vector<int64_t>> &members = H.members;
  const std::vector<int64_t> &prow = H.prow, &pcol = H.pcol;
  const std::vector<double> &pval = H.pval;
  const std::vector<uint8_t> &dir = H.dir;
  // P^T (CSR), each true dof's entries in ascending row order
  std::vector<int64_t> trow(H.n_true + 1, 0), tcol(pcol.size());
  std::vector<double> tval(pcol.size());
  for (int64_t c : pcol) trow[c + 1]++;
  for (int64_t i = 0; i < H.n_true; ++i) trow[i + 1] += trow[i];
  {
    std::vector<int64_t> fill(trow.begin(), trow.end() - 1);
    for (int64_t r = 0; r < rows; ++r)
      for (int64_t k = prow[r]; k < prow[r + 1]; ++k) {
        const int64_t q = fill[pcol[k]]++;
        tcol[q] = r;
        tval[q] = pval[k];
      }
  }
  int st;
  if ((st = upload(&h->d_prow, prow, s)) || (st = upload(&h->d_pcol, pcol, s)) || (st = upload(&h->d_pval, pval, s)) ||
      (st = upload(&h->d_trow, trow, s)) || (st = upload(&h->d_tcol, tcol, s)) || (st = upload(&h->d_tval, tval, s)) ||
      (st = upload(&h->d_dir, dir, s)))
    return st;
  CEED_CUDA_CHECK(cudaMalloc(&h->d_u, rows * sizeof(double)));
  CEED_CUDA_CHECK(cudaMalloc(&h->d_v, rows * sizeof(double)));

  // one mesh per order group whose nodes are the group's element vectors (identity restriction)
  std::vector<double> vert_all((size_t)E * 24);
  CEED_CUDA_CHECK(cudaMemcpyAsync(vert_all.data(), desc->vertices, vert_all.size() * 8, cudaMemcpyDeviceToHost, s));
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  for (size_t g = 0; g < porders.size(); ++g) {
    ceed_hp_s::Group &G = h->groups[g];
    const int64_t nd = (int64_t)(G.p + 1) * (G.p + 1) * (G.p + 1);
    std::vector<int32_t> ids(G.n_elem * nd);
    for (int64_t i = 0; i < (int64_t)ids.size(); ++i) ids[i] = (int32_t)i;
    std::vector<double> vs(G.n_elem * 24);
    for (int64_t i = 0; i < G.n_elem; ++i)
      std::memcpy(&vs[i * 24], &vert_all[members[g][i] * 24], 24 * sizeof(double));
    int32_t *d_ids = nullptr;
    double *d_vs = nullptr;
    if ((st = upload(&d_ids, ids, s)) != CEED_OK) return st;
    if ((st = upload(&d_vs, vs, s)) != CEED_OK) {
      cudaFree(d_ids);
      return st;
    }
    ceed_mesh_desc md;
    std::memset(&md, 0, sizeof(md));
    md.n_elem = G.n_elem;
    md.n_ldof = G.n_elem * nd;
    md.p = G.p;
    md.q_rule = h->q_rule;
    md.ncomp = 1;
    md.elem_dofs = d_ids;
    md.vertices = d_vs;
    st = ceed_setup_mesh(&md, &G.mesh, stream);
    cudaFree(d_ids);
    cudaFree(d_vs);
    if (st != CEED_OK) return st;
  }
  CEED_CUDA_CHECK(cudaStreamSynchronize(s));
  *out = h.release();
  return CEED_OK;
}

extern "C" int ceed_hp_destroy(ceed_hp_t h) {
  if (!h) return CEED_OK;
  cudaDeviceSynchronize();
  HpFree()(h);
  return CEED_OK;
}

extern "C" int ceed_hp_info(ceed_hp_t h, int64_t *n_true, int64_t *n_rows, int32_t *n_groups) {
  if (!h) return fail(CEED_ERR_INVALID, "null hp handle");
  if (n_true) *n_true = h->n_true;
  if (n_rows) *n_rows = h->n_rows;
  if (n_groups) *n_groups = (int32_t)h->groups.size();
  return CEED_OK;
}

static int hp_check(ceed_hp_t h, int op, int prec) {
  if (!h) return fail(CEED_ERR_INVALID, "null hp handle");
  if (op != CEED_OP_MASS && op != CEED_OP_DIFFUSION) return fail(CEED_ERR_INVALID, "op must be MASS or DIFFUSION");
  if (prec != CEED_F64 && prec != CEED_F32 && prec != CEED_F64_DF)
    return fail(CEED_ERR_UNSUPPORTED, "hp operator: prec F64, F32 or F64_DF");
  return CEED_OK;
}

// index of a precision in the groups' quadrature-data slots
static int hp_slot(int prec) { return prec == CEED_F64 ? 0 : prec == CEED_F32 ? 1 : 2; }

extern "C" int ceed_hp_build_qdata(ceed_hp_t h, int op, int coeff_kind, const double *coeff, int prec, void *stream) {
  int st = hp_check(h, op, prec);
  if (st != CEED_OK) return st;
  if (coeff_kind == CEED_COEFF_PER_QPT) return fail(CEED_ERR_UNSUPPORTED, "hp operator: per-point coefficients");
  const int pi = hp_slot(prec);
  for (auto &g : h->groups) {
    if (!g.qdata[op][pi]) {
      const size_t bytes = ceed_qdata_bytes(g.mesh, op, prec);
      CEED_CUDA_CHECK(cudaMalloc(&g.qdata[op][pi], bytes));
    }
    if ((st = ceed_build_qdata(g.mesh, op, coeff_kind, coeff, prec, g.qdata[op][pi], stream)) != CEED_OK) return st;
  }
  return CEED_OK;
}

extern "C" int ceed_hp_prolong(ceed_hp_t h, const double *x, double *u_elem, void *stream) {
  if (!h || !x || !u_elem) return fail(CEED_ERR_INVALID, "null hp handle or vector");
  cudaStream_t s = (cudaStream_t)stream;
  hp_spmv_kernel<<<(unsigned)((h->n_rows + 255) / 256), 256, 0, s>>>(h->n_rows, h->d_prow, h->d_pcol, h->d_pval, x,
                                                                      u_elem, h->d_dir, 0);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

extern "C" int ceed_hp_apply(ceed_hp_t h, int op, int prec, const double *x, double *y, unsigned flags, void *stream) {
  int st = hp_check(h, op, prec);
  if (st != CEED_OK) return st;
  if (!x || !y || x == y) return fail(CEED_ERR_INVALID, "null or overlapping x, y");
  const int pi = hp_slot(prec);
  for (auto &g : h->groups)
    if (!g.qdata[op][pi]) return fail(CEED_ERR_INVALID, "hp operator: quadrature data not built for this op/prec");
  const int masked = (flags & CEED_APPLY_DIRICHLET) && h->dirichlet;
  cudaStream_t s = (cudaStream_t)stream;
  hp_spmv_kernel<<<(unsigned)((h->n_rows + 255) / 256), 256, 0, s>>>(h->n_rows, h->d_prow, h->d_pcol, h->d_pval, x,
                                                                      h->d_u, h->d_dir, masked);
  CEED_CUDA_CHECK(cudaGetLastError());
  for (auto &g : h->groups) {
    st = op == CEED_OP_MASS
             ? ceed_apply_mass(g.mesh, g.qdata[op][pi], prec, h->d_u + g.row0, h->d_v + g.row0, 1, 0, stream)
             : ceed_apply_diffusion(g.mesh, g.qdata[op][pi], prec, h->d_u + g.row0, h->d_v + g.row0, 1, 0, stream);
    if (st != CEED_OK) return st;
  }
  hp_spmv_t_kernel<<<(unsigned)((h->n_true + 255) / 256), 256, 0, s>>>(h->n_true, h->d_trow, h->d_tcol, h->d_tval,
                                                                        h->d_v, x, y, h->d_dir, masked);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}
