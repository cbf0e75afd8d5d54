// pixel_groups.h -- host-side grouping of the detector pixels for the c-step.
//
// The compression merges the trilinear corners of neighbouring pixels before
// reducing them into the grid (compress.cu). Its groups: the pixels binned by
// cells of `cell` voxels in (q_x, q_y), in a stable order (pixel index within a
// cell), each cell's run cut into pieces of at most `max_group` pixels. A sheet
// of pixels (the Ewald-sphere slice, a graph over (q_x, q_y)) crosses each cell
// in a small patch, so a group's corners span a small box once rotated.
// Plain C++ (no CUDA), so the host tests compile it on its own.
#pragma once
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

namespace emc {

// q: double[n_pix][3] (voxel units). order receives the pixel indices in group
// order (n_pix entries); start the first position of every group followed by
// n_pix (ngroups + 1 entries).
inline void build_pixel_groups(const double* q, int64_t n_pix, double cell, int max_group,
                               std::vector<int32_t>& order, std::vector<int32_t>& start) {
  std::vector<int64_t> key(n_pix);
  for (int64_t i = 0; i < n_pix; i++) {
    const int64_t cx = (int64_t)floor(q[3 * i] / cell) + 4096;
    const int64_t cy = (int64_t)floor(q[3 * i + 1] / cell) + 4096;
    key[i] = cy * 16384 + cx;
  }
  order.resize(n_pix);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  start.clear();
  for (int64_t p = 0, run = 0; p < n_pix; p++) {
    if (p == 0 || key[order[p]] != key[order[p - 1]] || run == max_group) {
      start.push_back((int32_t)p);
      run = 0;
    }
    run++;
  }
  start.push_back((int32_t)n_pix);
}

}  // namespace emc
