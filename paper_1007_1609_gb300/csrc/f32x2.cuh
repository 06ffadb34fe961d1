// f32x2.cuh -- packed FP32 pairs for the fma.rn.f32x2 and sub.rn.f32x2
// instructions of sm_100 and later.  Each does two independent FP32
// operations with the rounding of the scalar instruction, so a sequence of
// packed operations gives, in each half, bit for bit the result of the same
// scalar sequence.  Used by the complex stencil (cplx_stencil.cuh).
#pragma once

namespace cbdg {

// lo = first float (the lower-addressed element of a float2 / float4 half)
using F2 = unsigned long long;
__device__ __forceinline__ F2 f2pack(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2unpack(F2 p, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ F2 f2fma(F2 a, F2 b, F2 c) {  // a * b + c, both halves, one rounding
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ F2 f2sub(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ F2 f2bcast(float x) { return f2pack(x, x); }
__device__ __forceinline__ F2 f2lo(const float4 &q) { return f2pack(q.x, q.y); }
__device__ __forceinline__ F2 f2hi(const float4 &q) { return f2pack(q.z, q.w); }

}  // namespace cbdg
