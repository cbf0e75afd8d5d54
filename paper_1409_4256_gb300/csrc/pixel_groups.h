// pixel_groups.h -- host-side grouping of the detector pixels for the c-step.
//
// The compression merges the trilinear corners of neighbouring pixels before
// reducing them into the grid (compress.cu); a warp takes one group, one pixel
// per lane. The groups come from a k-d split of the used pixels by (q_x, q_y):
// a set that holds more than `max_group` pixels, or spans more than
// `max_extent` voxels along q_x or q_y, is cut across its longer extent, so
// that the first part holds a multiple of `max_group` pixels (half of them,
// rounded, when the set is small enough but too wide). Every group but a few
// at the detector's edges and gaps is then full, and compact: a sheet of
// pixels (the Ewald-sphere slice, a graph over (q_x, q_y)) restricted to a
// small rectangle of (q_x, q_y) spans a small box of voxels once rotated.
// Groups follow the split's depth-first order; each keeps its pixels in index
// order. Plain C++ (no CUDA), so the host tests compile it on its own.
#pragma once
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <utility>
#include <vector>

namespace emc {

// q: double[n_pix][3] (voxel units, finite). order receives the pixel indices
// in group order (n_pix entries); start the first position of every group
// followed by n_pix (ngroups + 1 entries).
inline void build_pixel_groups(const double* q, int64_t n_pix, double max_extent, int max_group,
                               std::vector<int32_t>& order, std::vector<int32_t>& start) {
  order.resize(n_pix);
  std::iota(order.begin(), order.end(), 0);
  start.clear();
  // ranges [a, b) of `order` still to split, the next one on top
  std::vector<std::pair<int64_t, int64_t>> todo;
  if (n_pix > 0) todo.push_back({0, n_pix});
  while (!todo.empty()) {
    const int64_t a = todo.back().first, b = todo.back().second;
    todo.pop_back();
    const int64_t n = b - a;
    double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
    for (int64_t p = a; p < b; p++)
      for (int c = 0; c < 2; c++) {
        lo[c] = std::min(lo[c], q[3 * order[p] + c]);
        hi[c] = std::max(hi[c], q[3 * order[p] + c]);
      }
    const double ex = hi[0] - lo[0], ey = hi[1] - lo[1];
    if (n == 1 || (n <= max_group && ex <= max_extent && ey <= max_extent)) {
      std::sort(order.begin() + a, order.begin() + b);
      start.push_back((int32_t)a);
      continue;
    }
    const int c = ex >= ey ? 0 : 1;
    std::sort(order.begin() + a, order.begin() + b, [&](int32_t u, int32_t v) {
      const double qu = q[3 * u + c], qv = q[3 * v + c];
      return qu < qv || (qu == qv && u < v);
    });
    const int64_t k = n > max_group
                          ? (int64_t)max_group * (((n + max_group - 1) / max_group) / 2)
                          : n / 2;
    todo.push_back({a + k, b});  // the second part after the first
    todo.push_back({a, a + k});
  }
  start.push_back((int32_t)n_pix);
}

}  // namespace emc
