// FP64 <-> FP32 conversions with integer instructions only (GB300 runs conversions that involve
// FP64 on its narrow FP64 pipe; these keep the FP32 operators off it).
#pragma once

namespace ceedgb {

// FP64 -> FP32, round to nearest even, with integer instructions only.  Magnitudes below 2^-126
// flush to signed zero (FP32 denormals are not produced); Inf/NaN map to Inf/NaN; finite values of
// magnitude 2^128 and above become signed Inf, and values that round up past FLT_MAX carry into
// the Inf exponent, as IEEE rounding does.
__device__ __forceinline__ float d2f_int(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | ((hi & 0xfffffu) ? 0x400000u : 0u));
  if (e >= 1023 + 128) return __uint_as_float(sign | 0x7f800000u);
  if (e < 1023 - 126) return __uint_as_float(sign);
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  unsigned f = ((unsigned)(e - 1023 + 127) << 23) | mant;
  f += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | f);
}

// FP32 -> FP64 (exact), integer instructions only; FP32 denormals flush to zero.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi;
  if (e == 0) hi = sign;
  else if (e == 0xff) hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
  else hi = sign | ((e + (1023 - 127)) << 20) | (m >> 3);
  const unsigned lo = (e == 0) ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// Cheaper FP64 -> FP32 for the gather: a funnel shift brings the low 8 exponent bits and the top 23
// mantissa bits into float position; for the float range the double exponent is the float one plus
// 896 (= 3*256 + 128), so its low 8 bits differ from the float exponent only in the top bit (XOR).
// Rounds half up on the first dropped bit.  Magnitudes below 2^-126 give signed zero, Inf/NaN stay
// Inf/NaN, finite magnitudes of 2^128 and above saturate to signed Inf (a value rounding up past
// FLT_MAX carries into the Inf exponent by itself).
__device__ __forceinline__ float d2f_fast(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u, mag = hi & 0x7fffffffu;
  unsigned f = ((__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u) | sign;
  f += (lo >> 28) & 1u;
  f = (mag < 0x38100000u) ? sign : f;
  f = (mag >= 0x47f00000u) ? (sign | 0x7f800000u) : f;
  f = (mag >= 0x7ff00000u) ? (sign | 0x7f800000u | ((mag & 0xfffffu) | lo ? 0x400000u : 0u)) : f;
  return __uint_as_float(f);
}

// FP64 -> FP32 for a value that is exactly a float (written by f2d_int): no rounding, no range checks
// beyond zero.
__device__ __forceinline__ float d2f_exact(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const unsigned f = ((__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u) | sign;
  return __uint_as_float((hi & 0x7fffffffu) ? f : sign);
}

}  // namespace ceedgb
