// Phases of the Fourier-feature input layer gamma(p) (Sec. 4.3), shared by
// the FP32 and the 16-bit tensor-core kernels.
#pragma once

namespace nsdf {

// sin and cos of 2 pi (b . p) for a Fourier feature.  The FP32 product b . p
// would carry an absolute error of about ulp(b . p), which the 2 pi
// multiplies; instead the dot product is formed as an unevaluated sum hi + lo
// (the compensated dot product Dot2 of Ogita, Rump and Oishi, SIAM J. Sci.
// Comput. 26, 2005: error-free products by FMA, error-free sums by TwoSum),
// the nearest integer n of 2 hi is removed exactly, and sinpi / cospi of the
// small remainder are corrected by the sign (-1)^n.
__device__ __forceinline__ void ff_sincos(float bx, float by, float bz, float px, float py, float pz,
                                          float &sn, float &cs) {
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
  const float r = (yh - n) + 2.0f * lo;   // yh - n is exact
  sincospif(r, &sn, &cs);
  if (fabsf(n) < 16777216.0f && (static_cast<long long>(n) & 1LL)) {
    sn = -sn;
    cs = -cs;
  }
}

}  // namespace nsdf
