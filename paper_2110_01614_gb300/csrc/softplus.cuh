// FP32 softplus_beta and its slope on the special-function unit, shared by
// the tensor-core query kernels.
#pragma once

#include <cuda_runtime.h>

namespace nsdf {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;\n" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;\n" : "=f"(y) : "f"(x));
  return y;
}

// softplus_beta(z) and its slope sigmoid(beta z) from u = exp(-beta |z|):
//   softplus_beta(z) = max(z, 0) + log1p(u) / beta,
//   sigmoid(beta z)  = 1 / (1 + u) for z >= 0, u / (1 + u) otherwise.
// log1p(u) = u * P(u), P the degree-5 Chebyshev interpolant of log1p(u)/u on
// [0, 1] printed by gen_log1p_poly.py (relative error < 1e-5).  Two MUFU
// operations (ex2, rcp) per element; the rest runs on the FMA pipe.
// neg_bl2e = -beta * log2(e).
__device__ __forceinline__ void act_f32(float z, float neg_bl2e, float inv_beta, float &h,
                                        float &s) {
  const float u = ex2_approx(fabsf(z) * neg_bl2e);
  float p = -2.344365580e-02f;
  p = fmaf(p, u, 1.001397327e-01f);
  p = fmaf(p, u, -2.090795360e-01f);
  p = fmaf(p, u, 3.248495807e-01f);
  p = fmaf(p, u, -4.993146523e-01f);
  p = fmaf(p, u, 9.999905920e-01f);
  h = fmaf(u * p, inv_beta, fmaxf(z, 0.0f));
  const float r = rcp_approx(1.0f + u);
  s = (z >= 0.0f) ? r : u * r;
}

}  // namespace nsdf
