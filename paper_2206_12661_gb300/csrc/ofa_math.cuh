// Branch-free arg() for the phase projection of Algorithm 1 (phi = arg E').
//
// The octant is reduced with min/max and selects instead of branches, so the
// 32 lanes of a warp never diverge on the quadrant of their pixel:
//   a = min(|x|,|y|) / max(|x|,|y|) in [0, 1],  atan(a) = a P(a^2),
//   then pi/2 - r if |y| > |x|,  pi - r if x < 0,  and the sign of y.
// P is the degree-8 least-squares fit of atan(sqrt(t))/sqrt(t) on Chebyshev
// nodes of [0, 1] printed by gen_atan_poly.py in this directory; evaluated in
// FP32 its maximum absolute error on [0, 1] is 1.2e-7.  With the 2-ulp fast
// division the result is within about 3e-7 rad of atan2.  arg(0) = 0.
#pragma once

__device__ __forceinline__ float ofa_arg(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float hi = fmaxf(ax, ay), lo = fminf(ax, ay);
  const float a = hi > 0.f ? __fdividef(lo, hi) : 0.f;
  const float t = a * a;
  float p = 0.0028340642f;
  p = fmaf(p, t, -0.01600503f);
  p = fmaf(p, t, 0.042587608f);
  p = fmaf(p, t, -0.07495446f);
  p = fmaf(p, t, 0.10636754f);
  p = fmaf(p, t, -0.14202571f);
  p = fmaf(p, t, 0.19992484f);
  p = fmaf(p, t, -0.33333066f);
  p = fmaf(p, t, 1.0f);
  float r = a * p;                                   // atan(a), a in [0, 1]
  r = ay > ax ? 1.5707963267948966f - r : r;         // |y| > |x|: pi/2 - atan(x/y)
  r = x < 0.f ? 3.1415926535897932f - r : r;         // left half plane
  return copysignf(r, y);
}
