// Phases of the Fourier-feature input layer gamma(p) (Sec. 4.3), shared by
// the FP32 and the 16-bit tensor-core kernels.
#pragma once

#include <cstdint>

namespace nsdf {

// The reduced phase of a Fourier feature: 2 b.p = n + r with n an integer
// and |r| <= 1/2, so that sin(2 pi b.p) = (-1)^n sinpi(r) and likewise for
// cos; returns r and sets `odd` when n is odd.  The FP32
// product b . p would carry an absolute error of about ulp(b . p), which the
// 2 pi multiplies; instead the dot product is formed as an unevaluated sum
// hi + lo (the compensated dot product Dot2 of Ogita, Rump and Oishi, SIAM
// J. Sci. Comput. 26, 2005: error-free products by FMA, error-free sums by
// TwoSum), and the nearest integer n of 2 hi is removed exactly.
__device__ __forceinline__ float ff_reduced_phase(float bx, float by, float bz, float px, float py,
                                                  float pz, bool &odd) {
  const float p1 = bx * px, e1 = fmaf(bx, px, -p1);
  const float p2 = by * py, e2 = fmaf(by, py, -p2);
  const float p3 = bz * pz, e3 = fmaf(bz, pz, -p3);
  const float s12 = p1 + p2, v12 = s12 - p1;
  const float t12 = (p1 - (s12 - v12)) + (p2 - v12);
  const float hi = s12 + p3, v = hi - s12;
  const float t = (s12 - (hi - v)) + (p3 - v);
  const float lo = ((t12 + t) + e1) + (e2 + e3);
  const float yh = 2.0f * hi;
  const float n = rintf(yh);
  odd = fabsf(n) < 16777216.0f && (static_cast<long long>(n) & 1LL);
  return (yh - n) + 2.0f * lo;   // yh - n is exact
}

// sin and cos of 2 pi (b . p) in FP32: sinpi / cospi of the reduced phase.
__device__ __forceinline__ void ff_sincos(float bx, float by, float bz, float px, float py, float pz,
                                          float &sn, float &cs) {
  bool odd;
  const float r = ff_reduced_phase(bx, by, bz, px, py, pz, odd);
  sincospif(r, &sn, &cs);
  if (odd) {
    sn = -sn;
    cs = -cs;
  }
}

// sin and cos of 2 pi (b . p) for features that are rounded to a 16-bit
// format next (unit roundoff 2^-12 or coarser): y = 2 b.p by FMAs (absolute
// error a few ulp of |y|, about 2e-6 for |b.p| <= 16), the nearest integer n
// removed exactly, and sin / cos of pi r, |pi r| <= pi / 2, by the hardware
// approximations __sinf / __cosf (absolute error about 2^-21 on [-pi, pi]).
// The feature error stays near 1e-5, a twentieth of an FP16 ulp at
// |x| = 0.5; features that close to a rounding boundary of the format round
// the other way than the exact value would.  tb holds 2 b.
__device__ __forceinline__ void ff_sincos16(float tbx, float tby, float tbz, float px, float py,
                                            float pz, float &sn, float &cs) {
  const float y = fmaf(tbz, pz, fmaf(tby, py, tbx * px));
  const float n = rintf(y);
  const float a = 3.14159265358979324f * (y - n);   // y - n is exact
  sn = __sinf(a);
  cs = __cosf(a);
  if (fabsf(n) < 16777216.0f && (static_cast<int>(n) & 1)) {
    sn = -sn;
    cs = -cs;
  }
}

}  // namespace nsdf
