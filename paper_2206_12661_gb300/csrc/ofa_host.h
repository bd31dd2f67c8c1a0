// Host-side helpers of plan creation: plain C++ (no CUDA), in a header of their
// own so that they can be compiled and tested on a machine without a GPU.
#pragma once

#include <cmath>
#include <cstddef>

namespace ofa_host {

// Peak and energy (sum of squares, in FP64) of a pupil amplitude.  Returns false
// when a value is negative, infinite or NaN.  The sums run in eight interleaved
// lanes added in a fixed order at the end: the result is the same on every run,
// and differs from a serial sum only by rounding.
inline bool amplitude_stats(const float* a, size_t n, double* amax, double* energy) {
  constexpr int L = 8;
  double mx[L] = {}, mn[L] = {}, sq[L] = {};
  size_t i = 0;
  for (; i + L <= n; i += L)
    for (int l = 0; l < L; ++l) {
      const double v = a[i + l];
      mx[l] = v > mx[l] ? v : mx[l];
      mn[l] = v < mn[l] ? v : mn[l];
      sq[l] += v * v;
    }
  for (; i < n; ++i) {
    const double v = a[i];
    mx[0] = v > mx[0] ? v : mx[0];
    mn[0] = v < mn[0] ? v : mn[0];
    sq[0] += v * v;
  }
  double hi = 0.0, lo = 0.0, e = 0.0;
  for (int l = 0; l < L; ++l) {
    hi = mx[l] > hi ? mx[l] : hi;
    lo = mn[l] < lo ? mn[l] : lo;
    e += sq[l];
  }
  *amax = hi;
  *energy = e;
  // a NaN or an infinity makes the energy non-finite; a negative value the minimum
  return lo >= 0.0 && std::isfinite(e);
}

}  // namespace ofa_host
