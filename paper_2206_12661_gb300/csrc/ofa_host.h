// Host-side helpers of plan creation: plain C++ (no CUDA), in a header of their own so
// that they can be compiled and tested on a machine without a GPU.
#pragma once

#include <algorithm>
#include <cstddef>
#include <unordered_set>
#include <utility>
#include <vector>

namespace ofa_host {

// The distinct values of coordinate c (0: x, 1: y) of the n foci xy[n][2], sorted
// ascending, if there are at most lim of them; false (out unspecified) as soon as a
// (lim + 1)-th value appears, so a plan of scattered foci stops early.  Equal values
// count once (-0.0 and 0.0 are equal).
inline bool distinct_coords(const double* xy, int n, int c, size_t lim,
                            std::vector<double>& out) {
  std::unordered_set<double> seen;
  seen.reserve(std::min((size_t)n, lim + 1));
  for (int k = 0; k < n; ++k) {
    seen.insert(xy[2 * (size_t)k + c]);
    if (seen.size() > lim) return false;
  }
  out.assign(seen.begin(), seen.end());
  std::sort(out.begin(), out.end());
  return true;
}

// Whether no two of the n foci xy[n][2] sit on the same point (equal x and equal y).
inline bool one_focus_per_point(const double* xy, int n) {
  std::vector<std::pair<double, double>> pts(n);
  for (int k = 0; k < n; ++k) pts[k] = {xy[2 * (size_t)k], xy[2 * (size_t)k + 1]};
  std::sort(pts.begin(), pts.end());
  return std::adjacent_find(pts.begin(), pts.end()) == pts.end();
}

}  // namespace ofa_host
