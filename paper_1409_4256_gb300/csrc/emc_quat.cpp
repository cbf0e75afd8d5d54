// emc_quat.cpp -- rotation sampling of Eq. 2.7 (Sec. 2.2), host side.
//
// The 600-cell (120 vertices on the unit 3-sphere, 600 tetrahedral cells) is
// refined by dividing every cell n times: the lattice points
// sum_a (m_a / n) v_a (m_a >= 0, sum m_a = n) of all cells, merged where cells
// share faces, edges or vertices, are projected radially onto S^3. Opposite
// quaternions are the same rotation, so one of each pair is kept, leaving
// M_rot = 10 (5 n^3 + n) rotations.
//
// Prior weight w_j (the paper says only that the weights make the sampling
// practically uniform): the Jacobian of radial projection from a flat cell at
// distance r0 from the origin onto S^3 is r0 / |x|^4, so w_j ~ 1 / |x_j|^4 for
// the flat point x_j; weights are normalised to sum 1.
//
// Output order (an interface convention): sign fixed so that the first
// non-zero component is positive; k_c = round(q_c * 2^30); sorted by the
// 30-bit Morton code of the top 10 bits of k_x + 2^30, k_y + 2^30, k_z + 2^30
// (a space-filling curve through the rotations, so that consecutive indices --
// and 128-rotation tiles -- cover compact regions of SO(3)), ties broken by
// (k_w, k_x, k_y, k_z) lexicographically.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <unordered_set>
#include <vector>

#include "emc_internal.h"

namespace emc {
namespace {

using V4 = std::array<double, 4>;

std::vector<V4> vertices_600cell() {
  std::vector<V4> v;
  const double phi = 0.5 * (1.0 + std::sqrt(5.0));
  for (int a = 0; a < 4; a++)
    for (int s = -1; s <= 1; s += 2) {
      V4 x{0, 0, 0, 0};
      x[a] = s;
      v.push_back(x);
    }
  for (int m = 0; m < 16; m++) {
    V4 x;
    for (int c = 0; c < 4; c++) x[c] = ((m >> c) & 1) ? -0.5 : 0.5;
    v.push_back(x);
  }
  // even permutations of (phi, 1, 1/phi, 0) / 2 with all sign choices
  const double base[4] = {0.5 * phi, 0.5, 0.5 / phi, 0.0};
  int p[4] = {0, 1, 2, 3};
  std::sort(p, p + 4);
  do {
    int inv = 0;
    for (int a = 0; a < 4; a++)
      for (int b = a + 1; b < 4; b++) inv += p[a] > p[b];
    if (inv & 1) continue;
    for (int sg = 0; sg < 8; sg++) {
      V4 x{0, 0, 0, 0};
      for (int t = 0; t < 3; t++) x[p[t]] = ((sg >> t) & 1) ? -base[t] : base[t];
      x[p[3]] = 0.0;
      v.push_back(x);
    }
  } while (std::next_permutation(p, p + 4));
  return v;
}

struct KeyHash {
  size_t operator()(const std::array<int64_t, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t x : k) {
      h ^= (uint64_t)x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    }
    return (size_t)h;
  }
};

}  // namespace

int64_t quat_generate(int n, int uniform, double* quat, double* weight, int64_t cap) {
  if (n < 1 || n > 200) return EMC_ERR_ARG;
  const std::vector<V4> v = vertices_600cell();
  const int nv = (int)v.size();
  const double edge2 = (3.0 - std::sqrt(5.0)) / 2.0;  // (1/phi)^2
  std::vector<std::vector<int>> nb(nv);
  for (int a = 0; a < nv; a++)
    for (int b = 0; b < nv; b++) {
      if (a == b) continue;
      double d2 = 0;
      for (int c = 0; c < 4; c++) d2 += (v[a][c] - v[b][c]) * (v[a][c] - v[b][c]);
      if (std::fabs(d2 - edge2) < 1e-9) nb[a].push_back(b);
    }
  auto adj = [&](int a, int b) { return std::find(nb[a].begin(), nb[a].end(), b) != nb[a].end(); };
  std::vector<std::array<int, 4>> cells;
  for (int a = 0; a < nv; a++)
    for (int b : nb[a]) {
      if (b <= a) continue;
      for (int c : nb[a]) {
        if (c <= b || !adj(b, c)) continue;
        for (int d : nb[a]) {
          if (d <= c || !adj(b, d) || !adj(c, d)) continue;
          cells.push_back({a, b, c, d});
        }
      }
    }
  if (cells.size() != 600) return EMC_ERR_ARG;

  struct Rec {
    std::array<int64_t, 4> key;
    uint64_t code;
    V4 q;
    double w;
  };
  std::unordered_set<std::array<int64_t, 4>, KeyHash> seen;
  std::vector<Rec> out;
  const double scale = 1073741824.0;  // 2^30
  for (const auto& cell : cells)
    for (int m0 = 0; m0 <= n; m0++)
      for (int m1 = 0; m0 + m1 <= n; m1++)
        for (int m2 = 0; m0 + m1 + m2 <= n; m2++) {
          const int m3 = n - m0 - m1 - m2;
          const double m[4] = {(double)m0, (double)m1, (double)m2, (double)m3};
          V4 x{0, 0, 0, 0};
          for (int a = 0; a < 4; a++)
            for (int c = 0; c < 4; c++) x[c] += m[a] * v[cell[a]][c];
          for (int c = 0; c < 4; c++) x[c] /= n;
          // canonical sign: first component clearly away from zero is positive
          int sgn = 0;
          for (int c = 0; c < 4 && sgn == 0; c++)
            if (std::fabs(x[c]) > 1e-9) sgn = x[c] > 0 ? 1 : -1;
          if (sgn < 0) continue;  // the opposite point is generated by the opposite cell
          std::array<int64_t, 4> fk;
          for (int c = 0; c < 4; c++) fk[c] = std::llround(x[c] * scale);
          if (!seen.insert(fk).second) continue;
          double r2 = 0;
          for (int c = 0; c < 4; c++) r2 += x[c] * x[c];
          const double r = std::sqrt(r2);
          Rec rec;
          for (int c = 0; c < 4; c++) {
            rec.q[c] = x[c] / r;
            rec.key[c] = std::llround(rec.q[c] * scale);
          }
          rec.w = uniform ? 1.0 : 1.0 / (r2 * r2);
          out.push_back(rec);
        }
  auto morton = [](const std::array<int64_t, 4>& k) {
    uint64_t code = 0;
    for (int d = 0; d < 3; d++) {
      int64_t u = (k[1 + d] + (int64_t(1) << 30)) >> 21;  // 10 bits of [0, 2^31]
      u = u < 0 ? 0 : (u > 1023 ? 1023 : u);
      for (int b = 0; b < 10; b++) code |= (uint64_t)((u >> b) & 1) << (3 * b + d);
    }
    return code;
  };
  for (Rec& r : out) r.code = morton(r.key);
  std::sort(out.begin(), out.end(), [](const Rec& a, const Rec& b) {
    return a.code != b.code ? a.code < b.code : a.key < b.key;
  });
  const int64_t count = (int64_t)out.size();
  if (quat == nullptr && weight == nullptr) return count;
  if (count > cap) return EMC_ERR_ARG;
  double ws = 0;
  for (const Rec& r : out) ws += r.w;
  for (int64_t j = 0; j < count; j++) {
    if (quat)
      for (int c = 0; c < 4; c++) quat[4 * j + c] = out[j].q[c];
    if (weight) weight[j] = out[j].w / ws;
  }
  return count;
}

}  // namespace emc
