// Paired FP32 arithmetic: Blackwell executes add/sub/mul/fma.rn.f32x2 on a
// 64-bit register pair as one instruction (two independent FP32 lanes, each
// rounded as the scalar instruction would be).  Shared by the FP32 and the
// float-float kernels; a value is the pair (lo lane, hi lane) = (x, y).
#pragma once

#include <cuda_runtime.h>

namespace ssqcd {

typedef unsigned long long f32x2_t;


__device__ __forceinline__ f32x2_t pk2(float lo, float hi) {
  f32x2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(f32x2_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f32x2_t fma2(f32x2_t a, f32x2_t b, f32x2_t c) {
  f32x2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2_t mul2(f32x2_t a, f32x2_t b) {
  f32x2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2_t add2(f32x2_t a, f32x2_t b) {
  f32x2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2_t sub2(f32x2_t a, f32x2_t b) {
  f32x2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2_t swap2(f32x2_t z) {
  const float2 v = upk2(z);
  return pk2(v.y, v.x);
}
__device__ __forceinline__ f32x2_t neg2(f32x2_t z) {
  const float2 v = upk2(z);
  return pk2(-v.x, -v.y);
}

}  // namespace ssqcd
