// Fused matrix-free element kernel: gather (L->E), sum-factorized 1D contractions to the
// quadrature points, pointwise quadrature operator, transposed contractions, scatter-add (E->L).
//
// Paper Section 2: w_L = A_L u_L with A_L = block-diag(A^e), A^e = D^T G^e D; the 3D derivative
// is applied as 1D contractions u_r(r_i, s_j, t_k) = sum_m Dhat_im u_mjk (likewise along s, t) and
// G^e is six diagonal matrices G_rr ... G_tt.  Section 3 (cuda-gen): the whole operator in one
// kernel with no global temporaries.  Section 1: sum factorization, O(p^{d+1}) work per element.
//
// GB300 design (one thread block handles NE elements, Q x Q threads per element):
//  * the element's quadrature data block is staged into shared memory by one TMA bulk copy
//    (cp.async.bulk + mbarrier) issued at kernel entry, so it streams in while the gather and the
//    forward contractions run; for several columns (components x right-hand sides) it is read once;
//  * every global load of an element (restriction, x, and the old y of nodes already written by an
//    earlier colour) is issued up front, so an element pays one memory latency, not four;
//  * each 1D pass is done by "line owners": a thread holds a whole line of the tile in registers and
//    applies the 1D operator with the even-odd (centro-symmetry) decomposition, which replaces an
//    n x n product by two (n/2) x (n/2) products plus n folds/unfolds (48 instead of 64 operations
//    for n = 8) -- on GB300 the FP64 pipe is the limit of the FP64 operator, so this is the lever;
//  * tiles are stored with row pitch Q+1 so the three access patterns (r-lines, s-lines, t-columns)
//    are free of shared-memory bank conflicts for 4- and 8-byte words;
//  * the FP32 operator converts FP64 L-vector values to FP32 and back with integer instructions and
//    accumulates across colours in FP32, so it issues no FP64-pipe instruction at all;
//  * elements of one colour share no node: the scatter is a plain store for the first writer of a
//    node and a load-add-store for later colours (old value loaded up front): deterministic and
//    atomic-free.
#pragma once

#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>

#include "convert.cuh"
#include "df.cuh"
#include "internal.h"

namespace ceedgb {

// ------------------------------------------------------------------ storage conversions
__device__ __forceinline__ DF q_to(DF v, DF) { return v; }
__device__ __forceinline__ double q_to(double v, double) { return v; }
__device__ __forceinline__ float q_to(float v, float) { return v; }
__device__ __forceinline__ float q_to(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ float q_to(__half v, float) { return __half2float(v); }

template <typename T>
struct LVec;
template <>
struct LVec<DF> {     // FP64-accurate double-float operator: split on the way in, one FP64 add on the way out
  static __device__ __forceinline__ DF in(double v) {
    const float h = d2f_fast(v);
    return DF(h, d2f_fast(v - f2d_int(h)));
  }
  static __device__ __forceinline__ double out(DF v) { return f2d_int(v.hi) + f2d_int(v.lo); }
  static __device__ __forceinline__ double add(double old, DF v) { return (old + f2d_int(v.hi)) + f2d_int(v.lo); }
};
template <>
struct LVec<double> {  // FP64 operator: native
  static __device__ __forceinline__ double in(double v) { return v; }
  static __device__ __forceinline__ double out(double v) { return v; }
  static __device__ __forceinline__ double add(double old, double v) { return old + v; }
};
template <>
struct LVec<float> {   // FP32 operator: integer conversions, FP32 accumulation across colours
  static __device__ __forceinline__ float in(double v) { return d2f_fast(v); }
  static __device__ __forceinline__ double out(float v) { return f2d_int(v); }
  static __device__ __forceinline__ double add(double old, float v) { return f2d_int(d2f_exact(old) + v); }
};

// ------------------------------------------------------------------ TMA bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Asks the memory system to bring `bytes` (a multiple of 16, 16-byte aligned) at `src` into L2,
// without waiting and without touching shared memory or registers.
__device__ __forceinline__ void l2_prefetch_bulk(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bounded wait on phase `parity`: returns false if the copy did not land within WAIT_COPY_DEFAULT
// polls, or at once when give_up_now is set (failure-path tests).  The loop bound stays a
// compile-time constant: a run-time bound made the compiler keep ~40 more registers live in the
// element kernels (64 -> 108 for the staged FP32 operator).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, bool give_up_now = false) {
  const uint32_t a = smem_u32(bar);
  if (give_up_now) return false;
  for (int it = 0; it < WAIT_COPY_DEFAULT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// The same wait with a run-time bound.  Which form is faster depends on the element kernel: with the
// run-time bound the compiler gives the staged FP64 operator 128 registers and hoists its loads
// (7.67 against 7.44 GDOF/s at 64^3, p = 7, measured), while the FP32 operators run as fast with
// the compile-time bound at far fewer registers (staged FP32: 64 against 108).
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, uint32_t parity, int limit) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// ------------------------------------------------------------------ even-odd 1D operator
// out = M v for an NO x NI matrix with M[NO-1-i][NI-1-j] = S M[i][j] (S = +1 centro-symmetric,
// S = -1 centro-antisymmetric).  With e_j = v_j + v_{NI-1-j}, o_j = v_j - v_{NI-1-j} (j < NI/2):
//   out_i        =      sum_j E_ij e_j + sum_j O_ij o_j + M[i][mid] v_mid
//   out_{NO-1-i} = S * (sum_j E_ij e_j - sum_j O_ij o_j + M[i][mid] v_mid)
// with E = (M[i][j] + M[i][NI-1-j]) / 2, O = (M[i][j] - M[i][NI-1-j]) / 2; odd NO adds the middle row.
template <int NO, int NI, int S, typename T>
__device__ __forceinline__ void eo_apply(const EOMat<T> &M, const T *v, T *out) {
  constexpr int HI = NI / 2, HO = NO / 2;
  T e[HI > 0 ? HI : 1], o[HI > 0 ? HI : 1];
#pragma unroll
  for (int j = 0; j < HI; ++j) {
    e[j] = v[j] + v[NI - 1 - j];
    o[j] = v[j] - v[NI - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < HO; ++i) {
    T a = (NI & 1) ? M.cmid[i] * v[HI] : (T)0;
    T b = 0;
#pragma unroll
    for (int j = 0; j < HI; ++j) {
      a += M.E[i * EO_H + j] * e[j];
      b += M.O[i * EO_H + j] * o[j];
    }
    out[i] = a + b;
    out[NO - 1 - i] = (S > 0) ? (a - b) : (b - a);
  }
  if constexpr (NO & 1) {
    T c = (NI & 1) ? M.cc * v[HI] : (T)0;
#pragma unroll
    for (int j = 0; j < HI; ++j) c += M.rmid[j] * ((S > 0) ? e[j] : o[j]);
    out[HO] = c;
  }
}

constexpr int APPLY_MAX_THREADS = 256;
#ifndef APPLY_DF_MAX_REGS
#define APPLY_DF_MAX_REGS 128
#endif
constexpr int APPLY_MAX_NE = 32;

// g1 a + g2 b + g3 c and a + b + c: plain FMAs for float/double, compensated for double-float
template <typename T>
__device__ __forceinline__ T dot3(T g1, T a, T g2, T b, T g3, T c) {
  return g1 * a + g2 * b + g3 * c;
}
template <>
__device__ __forceinline__ DF dot3<DF>(DF g1, DF a, DF g2, DF b, DF g3, DF c) {
  DFAcc A = acc_first(g1, a);
  acc_mac(A, g2, b);
  acc_mac(A, g3, c);
  return acc_get(A);
}
// pointwise q u (mass operator): one FMA-able product, or the double-float product rounded once
template <typename T>
__device__ __forceinline__ T qmul(T q, T u) {
  return q * u;
}
template <>
__device__ __forceinline__ DF qmul<DF>(DF q, DF u) {
  return acc_get(acc_first(q, u));
}
template <typename T>
__device__ __forceinline__ T add3(T a, T b, T c) {
  return a + b + c;
}
template <>
__device__ __forceinline__ DF add3<DF>(DF a, DF b, DF c) {
  return df_add(df_add(a, b), c);
}

// Even-odd 1D operator in double-float: folds/unfolds by exact-sum additions, the two half-size
// products by compensated dot products (same algebra as the float/double version above).  Row i's
// two sums, A = sum_j E_ij e_j and B = sum_j O_ij o_j, are independent and take the same steps, so
// they run side by side in the two lanes of packed FP32 instructions (lane 0 = A, lane 1 = B).
// With an odd NI the middle input's term cmid_i v_mid ends A's sum; lane 1 adds 0 * 0 meanwhile,
// which leaves B unchanged.
template <int NO, int NI, int S>
__device__ __forceinline__ void eo_apply(const EOMat<DF> &M, const DF *v, DF *out) {
  constexpr int HI = NI / 2, HO = NO / 2;
  float2 eoh[HI > 0 ? HI : 1], eol[HI > 0 ? HI : 1];  // (e_j, o_j): high words, low words
#pragma unroll
  for (int j = 0; j < HI; ++j) {
    const DF e = df_add(v[j], v[NI - 1 - j]), o = df_sub(v[j], v[NI - 1 - j]);
    eoh[j] = make_float2(e.hi, o.hi);
    eol[j] = make_float2(e.lo, o.lo);
  }
#pragma unroll
  for (int i = 0; i < HO; ++i) {
    DFAcc2 AB = acc2_first(M.eo_hi[i * EO_H], M.eo_lo[i * EO_H], eoh[0], eol[0]);
#pragma unroll
    for (int j = 1; j < HI; ++j) acc2_mac(AB, M.eo_hi[i * EO_H + j], M.eo_lo[i * EO_H + j], eoh[j], eol[j]);
    if constexpr (NI & 1)
      acc2_mac(AB, make_float2(M.cmid[i].hi, 0.f), make_float2(M.cmid[i].lo, 0.f), make_float2(v[HI].hi, 0.f),
               make_float2(v[HI].lo, 0.f));
    const DF a(AB.s.x, AB.c.x), b(AB.s.y, AB.c.y);
    out[i] = df_add(a, b);
    out[NO - 1 - i] = (S > 0) ? df_sub(a, b) : df_sub(b, a);
  }
  if constexpr (NO & 1) {
    const DF e0(eoh[0].x, eol[0].x), o0(eoh[0].y, eol[0].y);
    DFAcc C = (NI & 1) ? acc_first(M.cc, v[HI]) : acc_first(M.rmid[0], (S > 0) ? e0 : o0);
    if (NI & 1) acc_mac(C, M.rmid[0], (S > 0) ? e0 : o0);
#pragma unroll
    for (int j = 1; j < HI; ++j) {
      const DF ej(eoh[j].x, eol[j].x), oj(eoh[j].y, eol[j].y);
      acc_mac(C, M.rmid[j], (S > 0) ? ej : oj);
    }
    out[HO] = acc_get(C);
  }
}

template <int Q>
constexpr int max_elems_per_block() {
  return (Q * Q >= APPLY_MAX_THREADS) ? 1 : (APPLY_MAX_THREADS / (Q * Q));
}

template <int Q>
constexpr int default_elems_per_block() {
  return (Q * Q >= 128) ? 1 : (128 / (Q * Q));
}

template <int Q>
constexpr int tile_words() {
  return Q * Q * (Q + 1);
}

// Quadrature data of one element, in bytes (16-byte multiple; the layout of qdata_estride).
template <int Q, int OP, typename TQ>
constexpr size_t qblock_bytes() {
  constexpr size_t n = (OP == CEED_OP_DIFFUSION) ? 6 * Q * Q * Q : (OP == OP_DIFF_GEO) ? GEO_COEFFS + Q * Q * Q : Q * Q * Q;
  return (n * sizeof(TQ) + 15) & ~(size_t)15;
}

// Shared memory of one element: staged quadrature data (if STAGE) + the tiles.
template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
constexpr size_t apply_elem_smem() {
  constexpr size_t qbytes = STAGE ? ((qblock_bytes<Q, OP, TQ>() + 127) & ~(size_t)127) : 0;
  constexpr int ntiles = (OP == CEED_OP_MASS) ? 2 : 3;
  constexpr size_t tbytes = ((size_t)ntiles * tile_words<Q>() * sizeof(T) + 127) & ~(size_t)127;
  return qbytes + tbytes;
}

// Tile index: (t, s, r) -> (t * Q + s) * (Q + 1) + r.
template <int Q>
__device__ __forceinline__ int tix(int t, int s, int r) {
  return (t * Q + s) * (Q + 1) + r;
}

// The element's operator from its node values u (one column of P nodes per node thread) to its
// node results yv, through the quadrature points: interpolation (Gauss) or identity (collocated),
// the derivative passes, the pointwise quadrature operator, the transposed passes.  Every thread of
// the element takes part (the passes use block barriers); wait_q() runs before the first read of the
// quadrature data sq.  Shared with the one-element-per-block-share kernel below and with the brick
// kernel (brick.cuh).
template <int P, int Q, int OP, typename T, typename TQ, typename WaitQ>
__device__ __forceinline__ void element_op(const OpTab<T> &tab, const T (&u)[P], T (&yv)[P], const TQ *sq, T *sa,
                                           T *sb, T *sc, int i, int j, bool node_thread, bool active,
                                           WaitQ &wait_q) {
  constexpr bool COLLOC = (P == Q);
  constexpr int NQ = Q * Q * Q;
  // ---- interpolate to the quadrature points (identity when collocated)
  T uq[Q];
  if constexpr (COLLOC) {
#pragma unroll
    for (int k = 0; k < Q; ++k) uq[k] = u[k];
  } else {
    if (node_thread) {  // t: column owners (r = i, s = j) hold the line in registers
      T w[Q];
      eo_apply<Q, P, 1>(tab.eB, u, w);
#pragma unroll
      for (int k = 0; k < Q; ++k) sa[tix<Q>(k, j, i)] = w[k];
    }
    __syncthreads();
    if (i < P) {        // s: owners (r = i, t = j)
      T v[P], w[Q];
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = sa[tix<Q>(j, m, i)];
      eo_apply<Q, P, 1>(tab.eB, v, w);
#pragma unroll
      for (int n = 0; n < Q; ++n) sb[tix<Q>(j, n, i)] = w[n];
    }
    __syncthreads();
    {                   // r: owners (s = i, t = j)
      T v[P], w[Q];
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = sb[tix<Q>(j, i, m)];
      eo_apply<Q, P, 1>(tab.eB, v, w);
#pragma unroll
      for (int n = 0; n < Q; ++n) sa[tix<Q>(j, i, n)] = w[n];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < Q; ++k) uq[k] = sa[tix<Q>(k, j, i)];
  }

  // ---- quadrature-point operator
  T w[Q];
  wait_q();  // quadrature data in place (staged copies: bounded wait)
  if constexpr (OP == CEED_OP_MASS) {
#pragma unroll
    for (int k = 0; k < Q; ++k) w[k] = active ? qmul(q_to(sq[(k * Q + j) * Q + i], T()), uq[k]) : (T)0;
  } else {
    T ut[Q];
    eo_apply<Q, Q, -1>(tab.eD, uq, ut);
    if constexpr (COLLOC) {
#pragma unroll
      for (int k = 0; k < Q; ++k) sa[tix<Q>(k, j, i)] = uq[k];
      __syncthreads();
    }  // non-collocated: sa already holds uq at these positions
    {  // r: owners (s = i, t = j)
      T v[Q], g[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = sa[tix<Q>(j, i, m)];
      eo_apply<Q, Q, -1>(tab.eD, v, g);
#pragma unroll
      for (int n = 0; n < Q; ++n) sb[tix<Q>(j, i, n)] = g[n];
    }
    {  // s: owners (r = i, t = j)
      T v[Q], g[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = sa[tix<Q>(j, m, i)];
      eo_apply<Q, Q, -1>(tab.eD, v, g);
#pragma unroll
      for (int n = 0; n < Q; ++n) sc[tix<Q>(j, n, i)] = g[n];
    }
    __syncthreads();
    // pointwise v = G grad u at my column, in place
    T vt[Q];
    // on-the-fly geometry: the trilinear map x = a0 + a1 r + a2 s + a3 t + a4 rs + a5 rt + a6 st + a7 rst
    // gives dx/dr = (a1 + a4 s) + (a5 + a7 s) t, dx/ds = (a2 + a4 r) + (a6 + a7 r) t and
    // dx/dt = a3 + a5 r + a6 s + a7 rs, so along my column only t varies: 6 FMAs per point for J
    T c1[3], c1t[3], c2[3], c2t[3], c3[3];
    if constexpr (OP == OP_DIFF_GEO) {
      const T xr = tab.qx[i], xs = tab.qx[j];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T a1 = q_to(sq[c], T()), a2 = q_to(sq[3 + c], T()), a3 = q_to(sq[6 + c], T());
        const T a4 = q_to(sq[9 + c], T()), a5 = q_to(sq[12 + c], T()), a6 = q_to(sq[15 + c], T());
        const T a7 = q_to(sq[18 + c], T());
        c1[c] = a1 + a4 * xs;
        c1t[c] = a5 + a7 * xs;
        c2[c] = a2 + a4 * xr;
        c2t[c] = a6 + a7 * xr;
        c3[c] = a3 + a5 * xr + a6 * xs + a7 * xr * xs;
      }
    }
    // double-float with an even number of points per column: points k and k + 1 share the two
    // lanes of the packed instructions (the same steps as dot3<DF>, lane by lane: bit-identical)
    constexpr bool PAIRED = std::is_same<T, DF>::value && OP == CEED_OP_DIFFUSION && (Q % 2 == 0);
    if constexpr (PAIRED) {
#pragma unroll
      for (int k = 0; k < Q; k += 2) {
        const int q0 = (k * Q + j) * Q + i, q1 = q0 + Q * Q;
        DF g0[6], g1[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          g0[c] = q_to(sq[c * NQ + q0], T());
          g1[c] = q_to(sq[c * NQ + q1], T());
        }
        const DF ur0 = sb[tix<Q>(k, j, i)], ur1 = sb[tix<Q>(k + 1, j, i)];
        const DF us0 = sc[tix<Q>(k, j, i)], us1 = sc[tix<Q>(k + 1, j, i)];
        const float2 urh = make_float2(ur0.hi, ur1.hi), url = make_float2(ur0.lo, ur1.lo);
        const float2 ush = make_float2(us0.hi, us1.hi), usl = make_float2(us0.lo, us1.lo);
        const float2 uth = make_float2(ut[k].hi, ut[k + 1].hi), utl = make_float2(ut[k].lo, ut[k + 1].lo);
        float2 gh[6], gl[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          gh[c] = make_float2(g0[c].hi, g1[c].hi);
          gl[c] = make_float2(g0[c].lo, g1[c].lo);
        }
        // components rr 0, rs 1, rt 2, ss 3, st 4, tt 5
        DFAcc2 A = acc2_first(gh[0], gl[0], urh, url);
        acc2_mac(A, gh[1], gl[1], ush, usl);
        acc2_mac(A, gh[2], gl[2], uth, utl);
        DFAcc2 B = acc2_first(gh[1], gl[1], urh, url);
        acc2_mac(B, gh[3], gl[3], ush, usl);
        acc2_mac(B, gh[4], gl[4], uth, utl);
        DFAcc2 C = acc2_first(gh[2], gl[2], urh, url);
        acc2_mac(C, gh[4], gl[4], ush, usl);
        acc2_mac(C, gh[5], gl[5], uth, utl);
        sb[tix<Q>(k, j, i)] = DF(A.s.x, A.c.x);
        sb[tix<Q>(k + 1, j, i)] = DF(A.s.y, A.c.y);
        sc[tix<Q>(k, j, i)] = DF(B.s.x, B.c.x);
        sc[tix<Q>(k + 1, j, i)] = DF(B.s.y, B.c.y);
        vt[k] = DF(C.s.x, C.c.x);
        vt[k + 1] = DF(C.s.y, C.c.y);
      }
    } else {
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int q = (k * Q + j) * Q + i;
      T grr, grs, grt, gss, gst, gtt;
      if constexpr (OP == OP_DIFF_GEO) {
        const T xt = tab.qx[k];
        T J[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          J[c][0] = c1[c] + c1t[c] * xt;
          J[c][1] = c2[c] + c2t[c] * xt;
          J[c][2] = c3[c];
        }
        // adjugate rows A_a (A J = det I) and G = (w k / det) A A^T
        const T A00 = J[1][1] * J[2][2] - J[1][2] * J[2][1], A01 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        const T A02 = J[0][1] * J[1][2] - J[0][2] * J[1][1], A10 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const T A11 = J[0][0] * J[2][2] - J[0][2] * J[2][0], A12 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        const T A20 = J[1][0] * J[2][1] - J[1][1] * J[2][0], A21 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        const T A22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const T det = J[0][0] * A00 + J[0][1] * A10 + J[0][2] * A20;
        const T f = active ? q_to(sq[GEO_COEFFS + q], T()) / det : (T)0;
        grr = f * (A00 * A00 + A01 * A01 + A02 * A02);
        grs = f * (A00 * A10 + A01 * A11 + A02 * A12);
        grt = f * (A00 * A20 + A01 * A21 + A02 * A22);
        gss = f * (A10 * A10 + A11 * A11 + A12 * A12);
        gst = f * (A10 * A20 + A11 * A21 + A12 * A22);
        gtt = f * (A20 * A20 + A21 * A21 + A22 * A22);
      } else {
        grr = q_to(sq[q], T()), grs = q_to(sq[NQ + q], T()), grt = q_to(sq[2 * NQ + q], T());
        gss = q_to(sq[3 * NQ + q], T()), gst = q_to(sq[4 * NQ + q], T()), gtt = q_to(sq[5 * NQ + q], T());
      }
      const T ur = sb[tix<Q>(k, j, i)], us = sc[tix<Q>(k, j, i)];
      sb[tix<Q>(k, j, i)] = dot3(grr, ur, grs, us, grt, ut[k]);
      sc[tix<Q>(k, j, i)] = dot3(grs, ur, gss, us, gst, ut[k]);
      vt[k] = dot3(grt, ur, gst, us, gtt, ut[k]);
    }
    }  // PAIRED
    __syncthreads();
    {  // r transposed: owners (s = i, t = j)
      T v[Q], g[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = sb[tix<Q>(j, i, m)];
      eo_apply<Q, Q, -1>(tab.eDT, v, g);
#pragma unroll
      for (int n = 0; n < Q; ++n) sa[tix<Q>(j, i, n)] = g[n];
    }
    {  // s transposed: owners (r = i, t = j), in place on their own line
      T v[Q], g[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = sc[tix<Q>(j, m, i)];
      eo_apply<Q, Q, -1>(tab.eDT, v, g);
#pragma unroll
      for (int n = 0; n < Q; ++n) sc[tix<Q>(j, n, i)] = g[n];
    }
    T yt[Q];
    eo_apply<Q, Q, -1>(tab.eDT, vt, yt);
    __syncthreads();
    if constexpr (PAIRED) {
#pragma unroll
      for (int k = 0; k < Q; k += 2) {  // add3 on points k and k + 1 together
        const DF a0 = sa[tix<Q>(k, j, i)], a1 = sa[tix<Q>(k + 1, j, i)];
        const DF c0 = sc[tix<Q>(k, j, i)], c1 = sc[tix<Q>(k + 1, j, i)];
        float2 h, l;
        df2_add(make_float2(yt[k].hi, yt[k + 1].hi), make_float2(yt[k].lo, yt[k + 1].lo),
                make_float2(a0.hi, a1.hi), make_float2(a0.lo, a1.lo), h, l);
        df2_add(h, l, make_float2(c0.hi, c1.hi), make_float2(c0.lo, c1.lo), h, l);
        w[k] = DF(h.x, l.x);
        w[k + 1] = DF(h.y, l.y);
      }
    } else {
#pragma unroll
      for (int k = 0; k < Q; ++k) w[k] = add3(yt[k], sa[tix<Q>(k, j, i)], sc[tix<Q>(k, j, i)]);
    }
  }

  // ---- transposed interpolation back to the nodes
  if constexpr (COLLOC) {
#pragma unroll
    for (int c = 0; c < P; ++c) yv[c] = w[c];
  } else {
    {  // t: column owners, registers
      T z[P];
      eo_apply<P, Q, 1>(tab.eBT, w, z);
      if constexpr (OP == CEED_OP_MASS) __syncthreads();  // sa was last read as the uq column
#pragma unroll
      for (int c = 0; c < P; ++c) sa[tix<Q>(c, j, i)] = z[c];
    }
    __syncthreads();
    if (j < P) {  // s: owners (r = i, t = j)
      T v[Q], z[P];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = sa[tix<Q>(j, m, i)];
      eo_apply<P, Q, 1>(tab.eBT, v, z);
#pragma unroll
      for (int n = 0; n < P; ++n) sb[tix<Q>(j, n, i)] = z[n];
    }
    __syncthreads();
    if (node_thread) {  // r: owners (s = i, t = j)
      T v[Q], z[P];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = sb[tix<Q>(j, i, m)];
      eo_apply<P, Q, 1>(tab.eBT, v, z);
#pragma unroll
      for (int n = 0; n < P; ++n) sa[tix<Q>(j, i, n)] = z[n];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < P; ++c) yv[c] = node_thread ? sa[tix<Q>(c, j, i)] : (T)0;
  }
}

struct ApplyArgs {
  const uint32_t *emap;
  const void *qdata;
  const double *x;
  double *y;
  int64_t e_begin, e_count;
  int64_t estride;  // quadrature data per element, in TQ units (16-byte multiple)
  int ncol, masked;
  int ne;           // elements per thread block
  int *err;
  int wait_limit;    // polls of the quadrature-data copy wait: 0 gives up at once (CEED_ERR_TIMEOUT), else
                     // the default bound
  double *dot_part;  // optional: partial sums of x_i y_i over the nodes whose final y this block writes
  int64_t dot_base;  // index of this launch's first block in dot_part
  double *dot_sh;    // optional, instead of dot_part: a shared-memory sum the block adds its partial to
                     // (thread 0, in the order the block processes its work: a persistent block's sum)
};

// One thread block's share of a colour: elements e_begin + blk * ne + (0 .. ne-1).  Threads past
// ne * Q^2 (a block shape that does not divide evenly) act as an inactive element; the caller
// provides shared memory for ceil(blockDim / Q^2) elements and the mbarrier array.
// XCG: x is read through L2 only (ld.global.cg) instead of the read-only path: required when x
// changes during the kernel (the persistent CG iteration updates p between its applies).
template <int P, int Q, int OP, typename T, typename TQ, bool STAGE, bool XCG = false>
__device__ __forceinline__ void apply_block(const ApplyArgs &a, const OpTab<T> &tab, int64_t blk,
                                            unsigned char *smem_raw, uint64_t *bar) {
  constexpr int NPT = Q * Q;
  constexpr int ND = P * P * P;
  constexpr size_t QB = STAGE ? ((qblock_bytes<Q, OP, TQ>() + 127) & ~(size_t)127) : 0;
  constexpr size_t EB = apply_elem_smem<P, Q, OP, T, TQ, STAGE>();

  const int tid = threadIdx.x;
  const int el = tid / NPT;
  const int ij = tid - el * NPT;
  const int i = ij % Q, j = ij / Q;
  const int64_t e = a.e_begin + blk * a.ne + el;
  const bool active = (el < a.ne) && (e < a.e_begin + a.e_count);
  const bool node_thread = (i < P) && (j < P);
  // staged block in shared memory, or the element's block in global memory
  const TQ *sq = STAGE ? (const TQ *)(smem_raw + el * EB) : (const TQ *)a.qdata + (active ? e : a.e_begin) * a.estride;
  T *sa = (T *)(smem_raw + el * EB + QB);
  T *sb = sa + tile_words<Q>();
  T *sc = sb + tile_words<Q>();  // diffusion only

  if constexpr (STAGE) {
    // ---- quadrature data: one bulk copy per element, in flight during the gather and the forward passes
    if (ij == 0) {
      mbar_init(&bar[el], 1);
      if (active)
        tma_bulk_load((void *)sq, (const TQ *)a.qdata + e * a.estride, (uint32_t)(a.estride * sizeof(TQ)), &bar[el]);
    }
    __syncthreads();  // barrier initialised before any thread waits on it
  } else {
    // quadrature data read at the pointwise step: start moving the element's block towards L2 now,
    // so that those loads wait for L2 rather than DRAM
    if (ij == 0 && active)
      l2_prefetch_bulk((const TQ *)a.qdata + e * a.estride, (uint32_t)(a.estride * sizeof(TQ)));
  }

  // ---- restriction of my node column (a = i, b = j, c = 0..P-1)
  uint32_t idx[P];
#pragma unroll
  for (int c = 0; c < P; ++c) idx[c] = 0;
  if (active && node_thread) {
    const uint32_t *em = a.emap + e * ND + j * P + i;
#pragma unroll
    for (int c = 0; c < P; ++c) idx[c] = __ldg(em + c * P * P);
  }
  bool have_q = false;
  bool q_ok = true;  // false once this thread's copy wait gave up: the element then writes nothing
  auto wait_q = [&]() {
    if (STAGE && !have_q) {  // elements past the end issued no copy and do not wait
      bool landed = true;
      if (active)
        landed = std::is_same<T, double>::value ? mbar_wait_n(&bar[el], 0, a.wait_limit)
                                                : mbar_wait(&bar[el], 0, a.wait_limit == 0);
      if (!landed) {
        q_ok = false;
        if (ij == 0) *a.err = CEED_ERR_TIMEOUT;
      }
      have_q = true;
    }
  };

  for (int col = 0; col < a.ncol; ++col) {
    // ---- all global loads of the column up front: x at my nodes, old y where an earlier colour wrote
    // (the double-float operator, whose element work is long and register-hungry, loads the old y
    // only at the scatter: holding it across the element would cost 2P registers of occupancy)
    constexpr bool EARLY_YOLD = !std::is_same<T, DF>::value;
    double xv[P], yold[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      xv[c] = 0.0;
      yold[c] = 0.0;
      if (active && node_thread) {
        const uint32_t v = idx[c];
        const int64_t o = (int64_t)(v & DOF_MASK) * a.ncol + col;
        const bool dir = a.masked && (v & FLAG_DIR);
        if (!dir) xv[c] = XCG ? __ldcg(a.x + o) : __ldg(a.x + o);
        if (EARLY_YOLD && !dir && !(v & FLAG_FIRST)) yold[c] = __ldcg(a.y + o);  // L2: written by an earlier colour
      }
    }
    T u[P];
#pragma unroll
    for (int c = 0; c < P; ++c) u[c] = LVec<T>::in(xv[c]);

    T yv[P];
    element_op<P, Q, OP, T, TQ>(tab, u, yv, sq, sa, sb, sc, i, j, node_thread, active, wait_q);

    // ---- scatter-add (E -> L), atomic-free
    const bool fused_dot = a.dot_part || a.dot_sh;
    if constexpr (!EARLY_YOLD) {
      if (active && node_thread && q_ok) {
#pragma unroll
        for (int c = 0; c < P; ++c) {
          const uint32_t v = idx[c];
          const int64_t o = (int64_t)(v & DOF_MASK) * a.ncol + col;
          if (!(a.masked && (v & FLAG_DIR)) && !(v & FLAG_FIRST)) yold[c] = __ldcg(a.y + o);
        }
      }
    }
    if (!fused_dot) {
      if (active && node_thread && q_ok) {
#pragma unroll
        for (int c = 0; c < P; ++c) {
          const uint32_t v = idx[c];
          const int64_t o = (int64_t)(v & DOF_MASK) * a.ncol + col;
          if (a.masked && (v & FLAG_DIR)) {
            if (v & FLAG_FIRST) a.y[o] = XCG ? __ldcg(a.x + o) : a.x[o];
          } else if (v & FLAG_FIRST) {
            a.y[o] = LVec<T>::out(yv[c]);
          } else {
            a.y[o] = LVec<T>::add(yold[c], yv[c]);
          }
        }
      }
    } else {
      // same scatter, and x . y over the nodes whose final value this thread writes (fused CG dot:
      // the last writer of a node adds x_i y_i; a masked Dirichlet node's first writer adds x_i^2)
      double dot = 0.0;
      if (active && node_thread && q_ok) {
#pragma unroll
        for (int c = 0; c < P; ++c) {
          const uint32_t v = idx[c];
          const int64_t o = (int64_t)(v & DOF_MASK) * a.ncol + col;
          if (a.masked && (v & FLAG_DIR)) {
            if (v & FLAG_FIRST) {
              const double out = XCG ? __ldcg(a.x + o) : a.x[o];
              a.y[o] = out;
              dot += out * out;
            }
          } else {
            const double out = (v & FLAG_FIRST) ? LVec<T>::out(yv[c]) : LVec<T>::add(yold[c], yv[c]);
            a.y[o] = out;
            if (v & FLAG_LAST) dot += (XCG ? __ldcg(a.x + o) : __ldg(a.x + o)) * out;  // reloaded: keeps xv dead early
          }
        }
      }
      // fixed-order block reduction: warp shuffles, then the warps in order
      __shared__ double dsum[APPLY_MAX_THREADS / 32];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, off);
      if ((tid & 31) == 0) dsum[tid >> 5] = dot;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += dsum[w];
        if (a.dot_sh) *a.dot_sh += t;
        else a.dot_part[a.dot_base + blk] = t;
      }
    }
    if (col + 1 < a.ncol) __syncthreads();
  }
  // the block must not exit while its copy may still be writing shared memory: an element whose
  // wait gave up (or that never reached the pointwise step) waits once more, with the default bound
  if (STAGE && (!have_q || !q_ok) && active) mbar_wait(&bar[el], 0);
  if constexpr (STAGE) {  // retire the barrier so the slot can be initialised again by the next block
    __syncthreads();
    if (ij == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar[el])) : "memory");
  }
}

template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
__global__ void __launch_bounds__(APPLY_MAX_THREADS)
apply_kernel(const ApplyArgs a, const OpTab<T> tab) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar[STAGE ? APPLY_MAX_NE : 1];
  apply_block<P, Q, OP, T, TQ, STAGE>(a, tab, blockIdx.x, smem_raw, bar);
}

// The double-float instantiations under a register cap: that operator is bound by latency
// (dependent compensated sums, quadrature-data loads), so it is given more resident warps to switch
// between instead of registers to hoist loads into (128: the best of 96..255 measured at p = 7).
// Blocks of at most APPLY_MAX_THREADS threads.
template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
__global__ void __maxnreg__(APPLY_DF_MAX_REGS) apply_kernel_capped(const ApplyArgs a, const OpTab<T> tab) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar[STAGE ? APPLY_MAX_NE : 1];
  apply_block<P, Q, OP, T, TQ, STAGE>(a, tab, blockIdx.x, smem_raw, bar);
}

}  // namespace ceedgb

#include "brick.cuh"

namespace ceedgb {

// Launch one kernel per colour for a fixed (P, Q, op, T, TQ) and variant (elements per block, staging).
template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
int launch_variant(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, int ne, cudaStream_t s) {
  const size_t smem = (size_t)ne * apply_elem_smem<P, Q, OP, T, TQ, STAGE>();
  constexpr bool CAPPED = std::is_same<T, DF>::value;
  const void *kfn;
  if constexpr (CAPPED) kfn = (const void *)apply_kernel_capped<P, Q, OP, T, TQ, STAGE>;
  else kfn = (const void *)apply_kernel<P, Q, OP, T, TQ, STAGE>;
  if (int st = ensure_dynamic_smem(kfn, smem)) return st;
  const dim3 block(Q * Q * ne);
  ApplyArgs a;
  a.emap = m->d_emap;
  a.qdata = r.qdata;
  a.x = r.x;
  a.y = r.y;
  a.ncol = r.ncol;
  a.masked = r.masked;
  a.ne = ne;
  a.err = m->d_err + 1;
  a.wait_limit = copy_wait_limit();
  a.estride = qdata_estride(OP, sizeof(TQ), Q);
  a.dot_part = (r.ncol == 1) ? r.dot_part : nullptr;
  a.dot_base = 0;
  a.dot_sh = nullptr;
  for (int c = 0; c < m->n_colors; ++c) {
    a.e_begin = m->color_start[c];
    const int64_t n = m->color_start[c + 1] - a.e_begin;
    if (n == 0) continue;
    a.e_count = n;
    const dim3 grid((unsigned)((n + ne - 1) / ne));
    if constexpr (CAPPED) apply_kernel_capped<P, Q, OP, T, TQ, STAGE><<<grid, block, smem, s>>>(a, tab);
    else apply_kernel<P, Q, OP, T, TQ, STAGE><<<grid, block, smem, s>>>(a, tab);
    a.dot_base += grid.x;
  }
  if (r.dot_n) *r.dot_n = a.dot_part ? a.dot_base : 0;
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

template <int P, int Q, int OP, typename T, typename TQ>
int launch_colours(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, cudaStream_t s) {
  int ne = r.ne, stage = r.stage;
  if (ne <= 0) {  // autotuned choice for this (op, precision), else the default
    const ApplyChoice &ch = m->tuned[r.op][r.prec];
    ne = ch.ne > 0 ? ch.ne : default_elems_per_block<Q>();
    stage = ch.ne > 0 ? ch.stage : 1;
  }
  if (stage >= 2) {  // brick kernel: FP32-pipe operators on a brick lattice, one column
    if constexpr (std::is_same<T, float>::value) {
      if (m->n_bricks > 0 && r.ncol == 1) {
        if (stage == 3) return launch_bricks<P, Q, OP, T, TQ, true>(m, tab, r, s);
        return launch_bricks<P, Q, OP, T, TQ, false>(m, tab, r, s);
      }
    }
    if (r.ne > 0) return fail(CEED_ERR_UNSUPPORTED, "brick kernel: needs a brick lattice, one column, an FP32-pipe operator");
    ne = default_elems_per_block<Q>();  // a tuned brick choice on a request the bricks cannot serve
    stage = 1;
  }
  if (ne > max_elems_per_block<Q>() || ne > APPLY_MAX_NE) return fail(CEED_ERR_INVALID, "elements per block too large");
  if (stage) return launch_variant<P, Q, OP, T, TQ, true>(m, tab, r, ne, s);
  return launch_variant<P, Q, OP, T, TQ, false>(m, tab, r, ne, s);
}

// Dispatch on (P, collocated?) for one (op, T, TQ).
template <int OP, typename T, typename TQ>
int dispatch_apply_op(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, cudaStream_t s) {
  if (((uintptr_t)r.qdata & 15) != 0) return fail(CEED_ERR_INVALID, "qdata must be 16-byte aligned");
  const bool colloc = (m->Q == m->P);
#define CEEDGB_CASE(PP)                                                                      \
  case PP:                                                                                  \
    return colloc ? launch_colours<PP, PP, OP, T, TQ>(m, tab, r, s)                         \
                  : launch_colours<PP, PP + 1, OP, T, TQ>(m, tab, r, s);
  switch (m->P) {
    CEEDGB_CASE(2)
    CEEDGB_CASE(3)
    CEEDGB_CASE(4)
    CEEDGB_CASE(5)
    CEEDGB_CASE(6)
    CEEDGB_CASE(7)
    CEEDGB_CASE(8)
    CEEDGB_CASE(9)
    default:
      return fail(CEED_ERR_UNSUPPORTED, "p outside 1..8");
  }
#undef CEEDGB_CASE
}

// Dispatch on (P, collocated?, op) for one (T, TQ) pair.
template <typename T, typename TQ>
int dispatch_apply(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, cudaStream_t s) {
  return r.op == CEED_OP_MASS ? dispatch_apply_op<CEED_OP_MASS, T, TQ>(m, tab, r, s)
                              : dispatch_apply_op<CEED_OP_DIFFUSION, T, TQ>(m, tab, r, s);
}

}  // namespace ceedgb
