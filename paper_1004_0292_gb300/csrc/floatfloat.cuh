// Float-float ("double-float") arithmetic for the shift vectors of the
// SSQCD_FP64_DFSHIFT precision.
//
// A real number is held as the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, a 48-bit significand (relative spacing 2^-48,
// 32x FP64's 2^-53) in the FP32 exponent range.  The arithmetic runs on the
// FP32 pipes, which on this GPU issue 64x the FP64 rate, and a complex
// element takes 16 bytes (re.hi, im.hi, re.lo, im.lo) -- the size of an FP64
// complex -- so a kernel that streams such vectors stays bound by memory
// instead of by the FP64 pipe.
//
// Built on two error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2): s = fl(a + b) and the exact
//     rounding error e with a + b = s + e, for any a, b;
//   TwoProduct via FMA (Dekker 1971; with a fused multiply-add the error
//     term is fma(a, b, -p)): p = fl(a b), e with a b = p + e.
// FastTwoSum (Dekker) is TwoSum for |a| >= |b| in three operations.
// These need IEEE round-to-nearest FP32 without reassociation, which nvcc
// keeps unless fast-math flags are given.
#pragma once

#include <cuda_runtime.h>

namespace ssqcd {
namespace ff {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// (ch + cl) + (u1h + u1l)(v1h + v1l) + (u2h + u2l)(v2h + v2l) in float-float.
// The two leading products and their sum with ch are formed exactly (TwoProduct,
// TwoSum); the cross terms u_h v_l + u_l v_h and the lo parts are gathered in
// one FP32 sum, whose terms are all ~2^-24 of the leading ones; a FastTwoSum
// renormalises.  The result is within a few units of 2^-48 (|c| + |u1 v1| +
// |u2 v2|) of the exact value.
__device__ __forceinline__ float2 fma2(float ch, float cl, float u1h, float u1l, float v1h, float v1l, float u2h,
                                       float u2l, float v2h, float v2l) {
  const float p1 = __fmul_rn(u1h, v1h);
  const float e1 = __fmaf_rn(u1h, v1h, -p1);
  const float p2 = __fmul_rn(u2h, v2h);
  const float e2 = __fmaf_rn(u2h, v2h, -p2);
  float s1, t1, s2, t2;
  two_sum(ch, p1, s1, t1);
  two_sum(s1, p2, s2, t2);
  float lo = __fadd_rn(__fadd_rn(cl, __fadd_rn(e1, e2)), __fadd_rn(t1, t2));
  lo = __fmaf_rn(u1h, v1l, lo);
  lo = __fmaf_rn(u1l, v1h, lo);
  lo = __fmaf_rn(u2h, v2l, lo);
  lo = __fmaf_rn(u2l, v2h, lo);
  float h, l;
  fast_two_sum(s2, lo, h, l);
  return make_float2(h, l);
}

// Complex float-float value: {re.hi, im.hi, re.lo, im.lo}.
using cff = float4;

// c + u v for complex float-float c, u, v.
__device__ __forceinline__ cff cfma(cff c, cff u, cff v) {
  const float2 re = fma2(c.x, c.z, u.x, u.z, v.x, v.z, -u.y, -u.w, v.y, v.w);
  const float2 im = fma2(c.y, c.w, u.x, u.z, v.y, v.w, u.y, u.w, v.x, v.z);
  return make_float4(re.x, im.x, re.y, im.y);
}

// Nearest float-float to an FP64 complex (hi = fl32(x), lo = fl32(x - hi);
// x - hi is exact in FP64).
__device__ __forceinline__ cff from_double2(double2 x) {
  const float hx = __double2float_rn(x.x), hy = __double2float_rn(x.y);
  const float lx = __double2float_rn(x.x - (double)hx), ly = __double2float_rn(x.y - (double)hy);
  return make_float4(hx, hy, lx, ly);
}

__device__ __forceinline__ double2 to_double2(cff x) {
  return make_double2((double)x.x + (double)x.z, (double)x.y + (double)x.w);
}

}  // namespace ff
}  // namespace ssqcd
