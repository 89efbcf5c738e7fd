// Double-float ("f32x2") arithmetic for an FP64-accurate operator computed on the FP32 pipe.
//
// GB300 issues about 60 FP32 FMAs for every FP64 FMA, so a value x is carried as an unevaluated sum
// hi + lo of two floats (about 48 significant bits) and every contraction sum_m M_m v_m is evaluated
// with the compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005):
// exact products by FMA (TwoProduct), exact partial sums by Knuth's TwoSum, and the rounding errors
// accumulated in a second float, which returns the sum as if computed in twice the working precision.
// The cross terms m_hi v_lo + m_lo v_hi enter the error accumulator by FMA.  Accuracy ~ 2^-47 of the
// input scale per contraction, versus 2^-53 for native FP64: enough for 1e-12 agreement with an FP64
// reference (measured: ~1e-14).
#pragma once

#include <cuda_runtime.h>

namespace ceedgb {

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr DF(int v) : hi((float)v), lo(0.f) {}
};

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

__device__ __forceinline__ DF df_norm(DF a) {
  float s, e;
  two_sum(a.hi, a.lo, s, e);
  return DF(s, e);
}

// Sums are left unnormalised (lo may exceed half an ulp of hi after cancellation): every later use
// multiplies lo by an FMA whose rounding error is 2^-24 of a quantity already 2^-24 below the inputs,
// so the absolute error stays ~2^-48 of the input scale; the value is only collapsed at the end
// (to FP64, where hi + lo is exact).
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return DF(s, e + (a.lo + b.lo));
}

__device__ __forceinline__ DF df_sub(DF a, DF b) {
  float s, e;
  two_sum(a.hi, -b.hi, s, e);
  return DF(s, e + (a.lo - b.lo));
}

// Dot2 accumulator: s holds the running float sum of the product high parts, c every rounding error.
struct DFAcc {
  float s, c;
};

// (products by __fmul_rn: the compiler may not contract them into a later addition, which would
// break the error-free transformations)
__device__ __forceinline__ void acc_mac(DFAcc &A, DF m, DF v) {
  const float p = __fmul_rn(m.hi, v.hi);
  float e = fmaf(m.hi, v.hi, -p);  // TwoProduct error, exact
  e = fmaf(m.hi, v.lo, e);
  e = fmaf(m.lo, v.hi, e);
  float t, q;
  two_sum(A.s, p, t, q);
  A.s = t;
  A.c += q + e;
}

// First term of a Dot2 sum: the exact product split (TwoProduct) and its cross terms, with no
// TwoSum against an empty accumulator.  Bit-identical to acc_mac on {0, 0} (TwoSum(0, p) = (p, 0)
// exactly), but the compiler cannot drop those additions itself (0 + x differs from x for x = -0).
__device__ __forceinline__ DFAcc acc_first(DF m, DF v) {
  const float p = __fmul_rn(m.hi, v.hi);
  float e = fmaf(m.hi, v.hi, -p);
  e = fmaf(m.hi, v.lo, e);
  e = fmaf(m.lo, v.hi, e);
  return DFAcc{p, e};
}

__device__ __forceinline__ DF acc_get(const DFAcc &A) { return DF(A.s, A.c); }

// y = sum_j M_j v_j over an NI-term row stored with stride 1 (used by the even-odd kernels).
template <int N>
__device__ __forceinline__ DF df_dot(const DF *m, const DF *v) {
  DFAcc A = acc_first(m[0], v[0]);
#pragma unroll
  for (int j = 1; j < N; ++j) acc_mac(A, m[j], v[j]);
  return acc_get(A);
}

// ---------------------------------------------------------------- two sums side by side
// The same Dot2 steps on two independent sums at once, one per lane of a float2, with the packed
// two-lane FP32 instructions of sm_100 and later (fma.rn.f32x2 and friends): each lane is rounded
// exactly as the scalar operation would be, and one instruction issues the work of two.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

struct DFAcc2 {
  float2 s, c;
};

// first term m v of both sums: (mh, ml) and (vh, vl) hold the two lanes' high and low words
__device__ __forceinline__ DFAcc2 acc2_first(float2 mh, float2 ml, float2 vh, float2 vl) {
  const float2 p = mul2(mh, vh);
  float2 e = fma2(mh, vh, neg2(p));  // TwoProduct error, exact
  e = fma2(mh, vl, e);
  e = fma2(ml, vh, e);
  return DFAcc2{p, e};
}

__device__ __forceinline__ void acc2_mac(DFAcc2 &A, float2 mh, float2 ml, float2 vh, float2 vl) {
  const float2 p = mul2(mh, vh);
  float2 e = fma2(mh, vh, neg2(p));
  e = fma2(mh, vl, e);
  e = fma2(ml, vh, e);
  const float2 t = add2(A.s, p);       // TwoSum(A.s, p), lane by lane
  const float2 z = sub2(t, A.s);
  const float2 q = add2(sub2(A.s, sub2(t, z)), sub2(p, z));
  A.s = t;
  A.c = add2(A.c, add2(q, e));
}

// df_add on two values at once: (ah, al) and (bh, bl) hold the lanes' high and low words.
__device__ __forceinline__ void df2_add(float2 ah, float2 al, float2 bh, float2 bl, float2 &sh, float2 &sl) {
  const float2 s = add2(ah, bh);  // TwoSum(ah, bh), lane by lane
  const float2 z = sub2(s, ah);
  const float2 e = add2(sub2(ah, sub2(s, z)), sub2(bh, z));
  sh = s;
  sl = add2(e, add2(al, bl));
}

// Host/device split of a double into the nearest float and the float nearest to the remainder.
__host__ __device__ inline DF df_from_double(double v) {
  const float h = (float)v;
  return DF(h, (float)(v - (double)h));
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

}  // namespace ceedgb
