// Paired FP32 arithmetic (f32x2) for the epilogues of the tensor-core
// kernels.
#pragma once

#include <cuda_runtime.h>

namespace nsdf {

// Two FP32 lanes per instruction (f32x2).  Each lane is the IEEE single
// result of the scalar operation with round-to-nearest, so these replace
// pairs of scalar FADD/FMUL/FFMA with identical values.  They also matter
// for speed beside the tensor cores: a stream of scalar FP32 FMA-pipe
// instructions on an SM slows the tcgen05 products issued there (measured
// with back-to-back M=128 N=256 products: 128 cycles each alone, 342 with
// eight warps of scalar FFMA, 128 with the same work in f32x2, HFMA2 or
// integer instructions).
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
      " add.rn.f32x2 d, a, b;\n mov.b64 {%0, %1}, d;\n}\n"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
      " mul.rn.f32x2 d, a, b;\n mov.b64 {%0, %1}, d;\n}\n"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// a * b + c per lane, one rounding
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 a, b, c, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
      " mov.b64 c, {%6, %7};\n fma.rn.f32x2 d, a, b, c;\n mov.b64 {%0, %1}, d;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 f2_splat(float v) { return make_float2(v, v); }

}  // namespace nsdf
