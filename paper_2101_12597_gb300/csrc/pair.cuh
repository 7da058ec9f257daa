// Float-pair numbers (hi, lo) held in a float2: the value is hi + lo, about 47
// significant bits in FP32's exponent range.  The mixed path's dense algebra
// runs on these: a pair multiply-add is about twelve FP32 operations, and FP32
// runs at more than sixty times the FP64 rate on this GPU.  Every operation is
// written with explicit round-to-nearest intrinsics, so that the compiler
// cannot contract the error-free transformations into fused forms that would
// break them.
#pragma once

#include <cuda_runtime.h>

namespace etdm {
namespace pair {

// s + e = a + b exactly (Knuth's TwoSum, six operations, no ordering needed)
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// h + l = a + b exactly when |a| >= |b| or a == 0 (Dekker's FastTwoSum)
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float h = __fadd_rn(a, b);
  return make_float2(h, __fsub_rn(b, __fsub_rn(h, a)));
}

__device__ __forceinline__ float2 add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);  // exact error of the high product
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return fast_two_sum(p, e);
}

// (h, l) += a b with the high parts' sum kept exactly (TwoSum) and the
// product's error, the cross terms and the sum's error gathered in l; l is
// left unnormalized (it stays below K ulp(h) after K steps).
__device__ __forceinline__ void mac(float &h, float &l, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float2 s = two_sum(h, p);
  l = __fadd_rn(l, __fadd_rn(s.y, e));
  h = s.x;
}

// multiplication by a power of two (exact unless it under- or overflows)
__device__ __forceinline__ float2 scale2(float2 a, float s) {
  return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
}

__device__ __forceinline__ double to_double(float2 a) { return (double)a.x + (double)a.y; }

// Split of an FP64 number into a float pair with integer operations only (no
// FP64 or conversion-pipe work): hi takes the leading 24 significand bits
// (truncated), lo the next 23, both exact, so |x - (hi + lo)| < 2^-46 |x|.
// Magnitudes below 2^-80 keep only hi (rounded), zero and subnormals give 0;
// values at or above 2^128 give +-inf in hi.
__device__ __forceinline__ float2 split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)(b >> 52) & 0x7ff;
  if (E == 0) return make_float2(0.f, 0.f);
  if (E < 943 || E > 1150) return make_float2(__double2float_rn(x), 0.f);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sgn | ((unsigned)(E - 896) << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
  // the next 23 bits as an integer (2^23 + r - 2^23 is exact), then its scale 2^(E-1069)
  const float r = __fsub_rn(__uint_as_float(0x4b000000u | ((unsigned)(b >> 6) & 0x7fffffu)), 8388608.f);
  const float lo = __fmul_rn(r, __uint_as_float((unsigned)(E - 942) << 23));
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sgn));
}

}  // namespace pair
}  // namespace etdm
