// Non-tensor operator handle, shared by the CUDA-core kernels (nontensor.cu) and the tensor-core
// kernel (nontensor_tc.cu).
#pragma once

#include <cublas_v2.h>

#include "internal.h"

namespace ceedgb {

constexpr int NT_MAXP = 128;   // basis functions per element
constexpr int NT_MAXQ = 1024;  // quadrature points per element
constexpr int NT_NE = 32;      // elements per block of the fused kernel (one per lane)
constexpr int NT_WARPS = 8;
constexpr int NT_QC = 32;      // quadrature points per chunk of the fused kernel
constexpr int NT_YR = NT_MAXP / NT_WARPS;

struct NtChoice {
  int algo = CEED_NT_FUSED;
  int64_t eta = 0;     // GEMM: elements per batched block (0: one GEMM over all elements)
  int gemm_mode = 0;   // GEMM: 0 native, 1 emulated on tensor cores, 2 TF32 (FP32 only)
  float ms = 0.f;
};

}  // namespace ceedgb

struct ceed_nt_s {
  int device = 0;
  int64_t E = 0, n_ldof = 0;
  int64_t Es = 0;              // element stride of the quadrature data: E rounded up to whole 128-element tiles
  int P = 0, Q = 0;
  double *d_tab64 = nullptr;   // [4][Q][P]: interp, then grad along xi_1, xi_2, xi_3
  float *d_tab32 = nullptr;
  ceedgb::DF *d_tabdf = nullptr;  // the same as double-float pairs (FP64-accurate fused kernel)
  double *d_qw = nullptr;      // [Q]
  double *d_qref = nullptr;    // [Q][3]
  uint32_t *d_rmap = nullptr;  // [P][E]
  int64_t *d_off = nullptr;    // [n_ldof + 1] transposed restriction offsets
  uint32_t *d_pos = nullptr;   // [P E] positions n E + e, ascending per node
  uint8_t *d_dir = nullptr;    // [n_ldof] Dirichlet flags (all zero without a mask)
  double *d_vert = nullptr;    // [E][4][3]
  int *d_err = nullptr;
  bool has_dirichlet = false;
  void *d_evec = nullptr;      // [P][E] element outputs (FP64-sized)
  void *d_u = nullptr;         // GEMM workspaces: [P][E] and [3 Q][E] (FP64-sized)
  void *d_s = nullptr;
  float *d_tc_tab[2] = {nullptr, nullptr};  // tensor-core tables per op (mass, diffusion), see nontensor_tc.cu
  int tc_nchunk = 0;
  cublasHandle_t blas = nullptr;
  ceedgb::NtChoice choice[2][3];  // [op][prec: 0 F64, 1 F32, 2 F64_DF (fused only)]
};

namespace ceedgb {
// Tensor-core (tcgen05) fused operator, FP32 accuracy by three TF32 products (nontensor_tc.cu).
bool nt_tc_supported(int P);
int nt_tc_prepare(ceed_nt_t h);   // builds the chunked split tables of both operators (once)
int nt_tc_apply(ceed_nt_t h, int op, const float *qd, const double *x, float *Ye, int masked, cudaStream_t s);
}  // namespace ceedgb
