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

#include "pair32.cuh"

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

// ---- real float-float values: float2 {hi, lo} --------------------------------

// a + b (two_sum of the leading parts, lo parts added, renormalised); the
// error is within a few units of 2^-48 (|a| + |b|).
__device__ __forceinline__ float2 add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  float h, l;
  fast_two_sum(s, e, h, l);
  return make_float2(h, l);
}

// c + u v
__device__ __forceinline__ float2 fma1(float2 c, float2 u, float2 v) {
  const float p = __fmul_rn(u.x, v.x);
  const float e = __fmaf_rn(u.x, v.x, -p);
  float s, t;
  two_sum(c.x, p, s, t);
  float lo = __fadd_rn(c.y, __fadd_rn(e, t));
  lo = __fmaf_rn(u.x, v.y, lo);
  lo = __fmaf_rn(u.y, v.x, lo);
  float h, l;
  fast_two_sum(s, lo, h, l);
  return make_float2(h, l);
}

// sum_i a_i b_i for K float-float pairs: the leading products and their sum
// exactly (TwoProduct, TwoSum chain), every lower-order term in one FP32
// sum, one renormalisation.
template <int K>
__device__ __forceinline__ float2 dot(const float2 (&a)[K], const float2 (&b)[K]) {
  float s = __fmul_rn(a[0].x, b[0].x);
  float lo = __fmaf_rn(a[0].x, b[0].x, -s);
  lo = __fmaf_rn(a[0].x, b[0].y, lo);
  lo = __fmaf_rn(a[0].y, b[0].x, lo);
#pragma unroll
  for (int i = 1; i < K; ++i) {
    const float p = __fmul_rn(a[i].x, b[i].x);
    const float e = __fmaf_rn(a[i].x, b[i].x, -p);
    float t;
    two_sum(s, p, s, t);
    lo = __fadd_rn(lo, __fadd_rn(e, t));
    lo = __fmaf_rn(a[i].x, b[i].y, lo);
    lo = __fmaf_rn(a[i].y, b[i].x, lo);
  }
  float h, l;
  fast_two_sum(s, lo, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }

// Nearest float-float to a double (x - hi is exact in FP64).
__device__ __forceinline__ float2 split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// Complex float-float value: {re.hi, im.hi, re.lo, im.lo}.
using cff = float4;

__device__ __forceinline__ float2 re(cff z) { return make_float2(z.x, z.z); }
__device__ __forceinline__ float2 im(cff z) { return make_float2(z.y, z.w); }
__device__ __forceinline__ cff make(float2 re_, float2 im_) { return make_float4(re_.x, im_.x, re_.y, im_.y); }
__device__ __forceinline__ cff cadd(cff a, cff b) { return make(add(re(a), re(b)), add(im(a), im(b))); }
__device__ __forceinline__ cff csub(cff a, cff b) { return make(add(re(a), neg(re(b))), add(im(a), neg(im(b)))); }
__device__ __forceinline__ cff cneg(cff a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
// exact scaling by a power of two
__device__ __forceinline__ cff cscale2(cff a, float s) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
// c + u v with u real
__device__ __forceinline__ cff caxpy(cff c, float2 u, cff v) { return make(fma1(re(c), u, re(v)), fma1(im(c), u, im(v))); }
// multiplication by +1, -1, +i, -i (codes 0..3): exact
__device__ __forceinline__ cff unit_mul(int code, cff z) {
  switch (code) {
    case 0: return z;
    case 1: return make_float4(-z.x, -z.y, -z.z, -z.w);
    case 2: return make_float4(-z.y, z.x, -z.w, z.z);
    default: return make_float4(z.y, -z.x, z.w, -z.z);
  }
}
// sum_b u_b h_b and sum_b conj(u_b) h_b over three complex float-float pairs
__device__ __forceinline__ cff cdot3(cff u0, cff u1, cff u2, cff h0, cff h1, cff h2) {
  const float2 ar[6] = {re(u0), neg(im(u0)), re(u1), neg(im(u1)), re(u2), neg(im(u2))};
  const float2 br[6] = {re(h0), im(h0), re(h1), im(h1), re(h2), im(h2)};
  const float2 ai[6] = {re(u0), im(u0), re(u1), im(u1), re(u2), im(u2)};
  const float2 bi[6] = {im(h0), re(h0), im(h1), re(h1), im(h2), re(h2)};
  return make(dot<6>(ar, br), dot<6>(ai, bi));
}
__device__ __forceinline__ cff cdot3_conj(cff u0, cff u1, cff u2, cff h0, cff h1, cff h2) {
  const float2 ar[6] = {re(u0), im(u0), re(u1), im(u1), re(u2), im(u2)};
  const float2 br[6] = {re(h0), im(h0), re(h1), im(h1), re(h2), im(h2)};
  const float2 ai[6] = {re(u0), neg(im(u0)), re(u1), neg(im(u1)), re(u2), neg(im(u2))};
  const float2 bi[6] = {im(h0), re(h0), im(h1), re(h1), im(h2), re(h2)};
  return make(dot<6>(ar, br), dot<6>(ai, bi));
}
// |z|^2 accumulated into a float-float sum (s, lo): exact squares of the
// leading parts, 2 hi lo cross terms in the FP32 low sum
__device__ __forceinline__ void norm2_acc(cff z, float& s, float& lo) {
  float p = __fmul_rn(z.x, z.x), t;
  lo = __fadd_rn(lo, __fmaf_rn(z.x, z.x, -p));
  two_sum(s, p, s, t);
  lo = __fadd_rn(lo, t);
  lo = __fmaf_rn(2.f * z.x, z.z, lo);
  p = __fmul_rn(z.y, z.y);
  lo = __fadd_rn(lo, __fmaf_rn(z.y, z.y, -p));
  two_sum(s, p, s, t);
  lo = __fadd_rn(lo, t);
  lo = __fmaf_rn(2.f * z.y, z.w, lo);
}

// c + u v for complex float-float c, u, v.
__device__ __forceinline__ cff cfma(cff c, cff u, cff v) {
  const float2 r_ = fma2(c.x, c.z, u.x, u.z, v.x, v.z, -u.y, -u.w, v.y, v.w);
  const float2 i_ = fma2(c.y, c.w, u.x, u.z, v.y, v.w, u.y, u.w, v.x, v.z);
  return make_float4(r_.x, i_.x, r_.y, i_.y);
}

// ---- complex float-float on register pairs -------------------------------------------
// A complex float-float value {re.hi, im.hi, re.lo, im.lo} is two register
// pairs: (re.hi, im.hi) and (re.lo, im.lo).  The real and imaginary parts of
// cadd, csub and the three-term complex dot products above run the same
// sequence of FP32 operations on different data, so they run here as one
// sequence of paired instructions (pair32.cuh), lane 0 the real part and
// lane 1 the imaginary part.  Every lane rounds exactly as the scalar code
// above does, in the same order: the results are bit-identical, with half
// the instructions.

__device__ __forceinline__ void p_two_sum(f32x2_t a, f32x2_t b, f32x2_t& s, f32x2_t& e) {
  s = ::ssqcd::add2(a, b);
  const f32x2_t bb = ::ssqcd::sub2(s, a);
  e = ::ssqcd::add2(::ssqcd::sub2(a, ::ssqcd::sub2(s, bb)), ::ssqcd::sub2(b, bb));
}
__device__ __forceinline__ void p_fast_two_sum(f32x2_t a, f32x2_t b, f32x2_t& s, f32x2_t& e) {
  s = ::ssqcd::add2(a, b);
  e = ::ssqcd::sub2(b, ::ssqcd::sub2(s, a));
}
__device__ __forceinline__ f32x2_t hi2(cff z) { return pk2(z.x, z.y); }
__device__ __forceinline__ f32x2_t lo2(cff z) { return pk2(z.z, z.w); }
__device__ __forceinline__ cff make2(f32x2_t h, f32x2_t l) {
  const float2 a = upk2(h), b = upk2(l);
  return make_float4(a.x, a.y, b.x, b.y);
}
// a + b and a - b (lane-wise float-float add of the real and imaginary parts)
__device__ __forceinline__ cff p_cadd(cff a, cff b) {
  f32x2_t s, e, h, l;
  p_two_sum(hi2(a), hi2(b), s, e);
  e = ::ssqcd::add2(e, ::ssqcd::add2(lo2(a), lo2(b)));
  p_fast_two_sum(s, e, h, l);
  return make2(h, l);
}
__device__ __forceinline__ cff p_csub(cff a, cff b) { return p_cadd(a, cneg(b)); }

// sum_i A_i B_i over K paired float-float factors (hi and lo pairs), the
// operation sequence of dot<K> in each lane
template <int K>
__device__ __forceinline__ cff p_dot(const f32x2_t (&ah)[K], const f32x2_t (&al)[K], const f32x2_t (&bh)[K],
                                     const f32x2_t (&bl)[K]) {
  f32x2_t s = ::ssqcd::mul2(ah[0], bh[0]);
  f32x2_t lo = ::ssqcd::fma2(ah[0], bh[0], neg2(s));
  lo = ::ssqcd::fma2(ah[0], bl[0], lo);
  lo = ::ssqcd::fma2(al[0], bh[0], lo);
#pragma unroll
  for (int i = 1; i < K; ++i) {
    const f32x2_t p = ::ssqcd::mul2(ah[i], bh[i]);
    const f32x2_t e = ::ssqcd::fma2(ah[i], bh[i], neg2(p));
    f32x2_t t;
    p_two_sum(s, p, s, t);
    lo = ::ssqcd::add2(lo, ::ssqcd::add2(e, t));
    lo = ::ssqcd::fma2(ah[i], bl[i], lo);
    lo = ::ssqcd::fma2(al[i], bh[i], lo);
  }
  f32x2_t h, l;
  p_fast_two_sum(s, lo, h, l);
  return make2(h, l);
}

// cdot3 / cdot3_conj on pairs: term 2b pairs (re u_b, re u_b) with
// (re h_b, im h_b), term 2b + 1 pairs (-im u_b, im u_b) (conj: (im u_b,
// -im u_b)) with (im h_b, re h_b) -- the factors of dot<6> in cdot3 for the
// real part (lane 0) and the imaginary part (lane 1).
// sg = -1: sum_b u_b h_b; sg = +1: sum_b conj(u_b) h_b (the direction of
// a hop may pick the sign at run time: the operations are the same)
__device__ __forceinline__ cff p_cdot3_sg(cff u0, cff u1, cff u2, cff h0, cff h1, cff h2, float sg) {
  const cff u[3] = {u0, u1, u2}, h[3] = {h0, h1, h2};
  f32x2_t ah[6], al[6], bh[6], bl[6];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    ah[2 * b] = pk2(u[b].x, u[b].x);
    al[2 * b] = pk2(u[b].z, u[b].z);
    ah[2 * b + 1] = pk2(sg * u[b].y, -sg * u[b].y);
    al[2 * b + 1] = pk2(sg * u[b].w, -sg * u[b].w);
    bh[2 * b] = hi2(h[b]);
    bl[2 * b] = lo2(h[b]);
    bh[2 * b + 1] = swap2(hi2(h[b]));
    bl[2 * b + 1] = swap2(lo2(h[b]));
  }
  return p_dot<6>(ah, al, bh, bl);
}
__device__ __forceinline__ cff p_cdot3(cff u0, cff u1, cff u2, cff h0, cff h1, cff h2) {
  return p_cdot3_sg(u0, u1, u2, h0, h1, h2, -1.f);
}
__device__ __forceinline__ cff p_cdot3_conj(cff u0, cff u1, cff u2, cff h0, cff h1, cff h2) {
  return p_cdot3_sg(u0, u1, u2, h0, h1, h2, 1.f);
}

// c + u v for complex float-float c, v and a coefficient u given as its four
// pairs U = {(u.re.hi, u.re.hi), (u.re.lo, u.re.lo), (-u.im.hi, u.im.hi),
// (-u.im.lo, u.im.lo)} (p_coef): the operation sequence of cfma in each lane.
struct PCoef {
  f32x2_t a1h, a1l, a2h, a2l;
};
__device__ __forceinline__ PCoef p_coef(cff u) {
  return PCoef{pk2(u.x, u.x), pk2(u.z, u.z), pk2(-u.y, u.y), pk2(-u.w, u.w)};
}
// v's pairs: (re.hi, im.hi), (re.lo, im.lo) and the same swapped
struct PVal {
  f32x2_t h, l, hs, ls;
};
__device__ __forceinline__ PVal p_val(cff v) {
  const f32x2_t h = hi2(v), l = lo2(v);
  return PVal{h, l, swap2(h), swap2(l)};
}
__device__ __forceinline__ void p_cfma(f32x2_t& ch, f32x2_t& cl, const PCoef& u, const PVal& v) {
  const f32x2_t p1 = ::ssqcd::mul2(u.a1h, v.h);
  const f32x2_t e1 = ::ssqcd::fma2(u.a1h, v.h, neg2(p1));
  const f32x2_t p2 = ::ssqcd::mul2(u.a2h, v.hs);
  const f32x2_t e2 = ::ssqcd::fma2(u.a2h, v.hs, neg2(p2));
  f32x2_t s1, t1, s2, t2;
  p_two_sum(ch, p1, s1, t1);
  p_two_sum(s1, p2, s2, t2);
  f32x2_t lo = ::ssqcd::add2(::ssqcd::add2(cl, ::ssqcd::add2(e1, e2)), ::ssqcd::add2(t1, t2));
  lo = ::ssqcd::fma2(u.a1h, v.l, lo);
  lo = ::ssqcd::fma2(u.a1l, v.h, lo);
  lo = ::ssqcd::fma2(u.a2h, v.ls, lo);
  lo = ::ssqcd::fma2(u.a2l, v.hs, lo);
  p_fast_two_sum(s2, lo, ch, cl);
}

// c + u v for a REAL float-float coefficient u, given as the pairs
// (u.hi, u.hi) and (u.lo, u.lo), and a complex float-float v: the real and
// imaginary parts are two independent float-float multiply-adds, one in
// each lane (the operation order of ff::fma1 on each part).
__device__ __forceinline__ void p_rfma(f32x2_t& ch, f32x2_t& cl, f32x2_t uh, f32x2_t ul, const PVal& v) {
  const f32x2_t p = ::ssqcd::mul2(uh, v.h);
  const f32x2_t e = ::ssqcd::fma2(uh, v.h, neg2(p));
  f32x2_t s, t;
  p_two_sum(ch, p, s, t);
  f32x2_t lo = ::ssqcd::add2(cl, ::ssqcd::add2(e, t));
  lo = ::ssqcd::fma2(uh, v.l, lo);
  lo = ::ssqcd::fma2(ul, v.h, lo);
  p_fast_two_sum(s, lo, ch, cl);
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
