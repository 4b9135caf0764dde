// FP32 softplus_beta and its slope on the special-function unit, shared by
// the tensor-core query kernels.
#pragma once

#include <cuda_runtime.h>

#include "f32x2.cuh"

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

// act_f32 for two elements at once (the same operations per lane, so the
// same values): softplus_beta(z) in h and its slope in s.
__device__ __forceinline__ void act_f32x2(float2 z, float neg_bl2e, float inv_beta, float2 &h,
                                          float2 &s) {
  const float2 az = make_float2(__uint_as_float(__float_as_uint(z.x) & 0x7fffffffu),
                                __uint_as_float(__float_as_uint(z.y) & 0x7fffffffu));
  const float2 t = f2_mul(az, f2_splat(neg_bl2e));
  const float2 u = make_float2(ex2_approx(t.x), ex2_approx(t.y));
  float2 p = f2_splat(-2.344365580e-02f);
  p = f2_fma(p, u, f2_splat(1.001397327e-01f));
  p = f2_fma(p, u, f2_splat(-2.090795360e-01f));
  p = f2_fma(p, u, f2_splat(3.248495807e-01f));
  p = f2_fma(p, u, f2_splat(-4.993146523e-01f));
  p = f2_fma(p, u, f2_splat(9.999905920e-01f));
  h = f2_fma(f2_mul(u, p), f2_splat(inv_beta), make_float2(fmaxf(z.x, 0.0f), fmaxf(z.y, 0.0f)));
  const float2 d = f2_add(f2_splat(1.0f), u);
  const float2 r = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  const float2 ur = f2_mul(u, r);
  s = make_float2(z.x >= 0.0f ? r.x : ur.x, z.y >= 0.0f ? r.y : ur.y);
}

}  // namespace nsdf
