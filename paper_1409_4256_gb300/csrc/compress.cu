// compress.cu -- c-step of EMC (Eq. 2.12; Eq. 2.5 + 2.10 in IDW mode).
//
// One CTA per rotation row j. Each (i, j) recomputes the grid point
// p = R_j q_i + N/2 (in fixed point, rotate_fx: the weights f(p_l - R_j q_i)
// of the expansion) and contributes f * Num_ij to g_num and f * den_j to
// g_den, which are
// reduced with FP64 atomics resolved in L2 (the N^3 FP64 grids, 2 MB at 64^3,
// stay L2-resident). The paper's insert_slices kernel also used one block per
// slice. Rotations without responsibility mass (den_j = 0) are skipped. Every
// slice passes through the centre of the grid, so concurrent CTAs reduce into
// the same central voxels; with nrep > 1 the CTA of row j uses grid replica
// j mod nrep (nrep x N^3 per grid, summed by the final division) to spread
// those reductions over more addresses.
//
// Corner merging. The used pixels are split by (q_x, q_y) into groups of at
// most 32 (pixel_groups.h), so a group is a small patch of the detector sheet,
// and neighbouring pixels share most of their trilinear corners (about 8
// corner terms per 3.3 distinct voxels). A warp takes one group (one pixel per
// lane; nearly every group is full, so few lanes idle), bounds its
// corners by a box, and sums the terms per voxel in a shared-memory box of
// FP32 pairs (numerator, denominator) before one FP64 reduction per touched
// voxel:
//  * pixels with the same floor cell share all eight voxels; __match_any_sync
//    finds them and the lowest lane sums their terms in lane order;
//  * the remaining lanes have distinct floor cells, so for one corner offset c
//    their voxels are distinct: corner by corner (a __syncwarp between
//    corners) each lane adds into its slot without atomics;
//  * the warp then sweeps the box in slot order: each non-zero slot is reduced
//    once and cleared. Consecutive lanes hold consecutive slots (neighbouring
//    z of one (x, y) column), so the sweep's loads are conflict-free and its
//    reductions touch few sectors per instruction.
// The order of every FP32 addition is fixed, so the result does not depend on
// scheduling beyond the FP64 order of the L2 reductions. A group whose box
// exceeds kAggCap slots reduces its corners directly.
#include <limits.h>

#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

constexpr int kAggWarps = 4;
constexpr int kAggCap = 576;       // box slots per warp (float2 each), below 1024
constexpr int kAggStage = 32 * 8;  // merge staging: 8 corner terms per lane
constexpr int kAggThreads = kAggWarps * 32;
// 26.6 KB per CTA: eight CTAs (32 warps) per SM, at most 64 registers a thread
constexpr size_t kAggSmem = sizeof(float2) * kAggWarps * (kAggCap + kAggStage);
static_assert(kCompressGroup == 32, "one pixel per lane");

__device__ __forceinline__ bool in_grid(int x, int y, int z, int N) {
  return (unsigned)x < (unsigned)N && (unsigned)y < (unsigned)N && (unsigned)z < (unsigned)N;
}

// the eight corner terms of one pixel straight into the grids
template <bool INTERIOR>
__device__ __forceinline__ void reduce_direct(const int* f, const float* t, float v, float dvi,
                                              int N, double* g_num, double* g_den) {
  const int64_t nn = (int64_t)N * N;
#pragma unroll
  for (int c = 0; c < 8; c++) {
    const int cx = (c >> 2) & 1, cy = (c >> 1) & 1, cz = c & 1;
    const int x = f[0] + cx, y = f[1] + cy, z = f[2] + cz;
    if (!INTERIOR && !in_grid(x, y, z, N)) continue;
    const float w = (cx ? t[0] : 1.f - t[0]) * (cy ? t[1] : 1.f - t[1]) * (cz ? t[2] : 1.f - t[2]);
    if (w == 0.f) continue;
    const int64_t l = (int64_t)x * nn + (int64_t)y * N + z;
    // FP32 products (relative error 6e-8), FP64 accumulation in L2
    atomicAdd(g_num + l, (double)(w * v));
    if (dvi != 0.f) atomicAdd(g_den + l, (double)(w * dvi));
  }
}

// warp-wide integer minimum and maximum: one redux instruction each (a
// butterfly of shuffles costs five shuffles, which share the load/store
// pipe's wavefronts with the box's shared-memory traffic)
__device__ __forceinline__ int warp_min(int v) { return __reduce_min_sync(0xffffffffu, v); }
__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(0xffffffffu, v); }

// INTERIOR: all trilinear corners of every pixel lie inside the grid (checked
// on the host from max |q_i|), so no bounds checks.
template <bool INTERIOR>
__global__ void __launch_bounds__(kAggThreads, 8)
    compress_kernel(Geom g, const RotFX* __restrict__ rot, const float* __restrict__ Num,
                    const float* __restrict__ den, int mode, double* __restrict__ g_num,
                    double* __restrict__ g_den, int nrep, int64_t n_vox) {
  extern __shared__ float2 agg_smem[];
  const int64_t row = blockIdx.x;
  const float dj = den[row];
  // a rotation without responsibility mass has Num = 0 and den = 0 (both
  // modes): it adds nothing, and sparse iterations leave most rows so
  if (!(dj > 0.f)) return;
  const int64_t rep = (row % nrep) * n_vox;
  g_num += rep;
  g_den += rep;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* box = agg_smem + warp * (kAggCap + kAggStage);
  float2* stage = box + kAggCap;
  // the row's rotation in registers (uniform loads, once per CTA)
  int Rh[9];
  float Rhf[9], Rl[9];
#pragma unroll
  for (int e = 0; e < 9; e++) {
    Rh[e] = __ldg(&rot[row].hi[e]);
    Rhf[e] = (float)Rh[e] * 0x1p-20f;
    Rl[e] = __ldg(&rot[row].lo[e]);
  }
  for (int s = lane; s < kAggCap; s += 32) box[s] = make_float2(0.f, 0.f);
  __syncwarp();
  const int N = g.N;
  const int64_t nn = (int64_t)N * N;
  const float* Nr = Num + row * g.ld_pix;
  const float inv_d = (mode == EMC_COMPRESS_IDW) ? 1.0f / dj : 1.0f;
  const float dv = (mode == EMC_COMPRESS_IDW) ? 1.0f : dj;

  for (int grp = warp; grp < g.ngroups; grp += kAggWarps) {
    const int p0 = g.gstart[grp], np = g.gstart[grp + 1] - p0;
    int f[3];
    float t[3], v;
    const bool has = lane < np;
    if (has) {
      rotate_fx(Rh, Rhf, Rl, g.gqi[p0 + lane], g.gqf[p0 + lane], g.gqlo[p0 + lane], N, f, t);
      v = Nr[g.gpix[p0 + lane]] * inv_d;
    } else {
      f[0] = f[1] = f[2] = 0;
      t[0] = t[1] = t[2] = 0.f;
      v = 0.f;
    }
    // the box of every corner of the group: floors lo .. hi, corners to hi + 1
    int lo[3], dim[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      lo[a] = warp_min(has ? f[a] : INT_MAX);
      dim[a] = warp_max(has ? f[a] : INT_MIN) - lo[a] + 2;
    }
    const int64_t vol = (int64_t)dim[0] * dim[1] * dim[2];
    if (vol > kAggCap) {
      if (has) reduce_direct<INTERIOR>(f, t, v, dv, N, g_num, g_den);
      continue;
    }
    // slot of corner 0; absent lanes get distinct negative keys
    const int key = has ? ((f[0] - lo[0]) * dim[1] + (f[1] - lo[1])) * dim[2] + (f[2] - lo[2])
                        : -1 - lane;
    const unsigned m = __match_any_sync(0xffffffffu, key);
    const bool lead = has && (__ffs(m) - 1 == lane);
    float2 acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      const int cx = (c >> 2) & 1, cy = (c >> 1) & 1, cz = c & 1;
      const float w = (cx ? t[0] : 1.f - t[0]) * (cy ? t[1] : 1.f - t[1]) *
                      (cz ? t[2] : 1.f - t[2]);
      acc[c] = make_float2(w * v, w * dv);
    }
    // pixels sharing a floor cell: the lowest lane sums the terms in lane order
    const bool shared = has && m != (1u << lane);
    if (__any_sync(0xffffffffu, shared)) {
      if (shared && !lead)
#pragma unroll
        for (int c = 0; c < 8; c++) stage[lane * 8 + c] = acc[c];
      __syncwarp();
      if (shared && lead) {
        unsigned rest = m & ~(1u << lane);
        while (rest) {
          const int l = __ffs(rest) - 1;
          rest &= rest - 1;
#pragma unroll
          for (int c = 0; c < 8; c++) {
            const float2 o = stage[l * 8 + c];
            acc[c].x += o.x;
            acc[c].y += o.y;
          }
        }
      }
      __syncwarp();
    }
    // corner by corner: the leaders' slots for one offset are distinct
#pragma unroll
    for (int c = 0; c < 8; c++) {
      const int cx = (c >> 2) & 1, cy = (c >> 1) & 1, cz = c & 1;
      if (lead && (INTERIOR || in_grid(f[0] + cx, f[1] + cy, f[2] + cz, N))) {
        const int s = key + (cx * dim[1] + cy) * dim[2] + cz;
        float2 b = box[s];
        b.x += acc[c].x;
        b.y += acc[c].y;
        box[s] = b;
      }
      __syncwarp();
    }
    // sweep the box in slot order: one reduction per non-zero slot. Slot
    // s = (x dim1 + y) dim2 + z; the quotients by multiply and shift with
    // m = ceil(2^20 / d): floor(s m / 2^20) = floor(s / d) for s < 1024,
    // since s (m - 2^20 / d) / 2^20 < 2^-10 < 1/d for d <= kAggCap. (Integer
    // arithmetic: conversions between int and float run on the FP64 pipe here.)
    const int d12 = dim[1] * dim[2];
    const unsigned m12 = ((1u << 20) + (unsigned)d12 - 1u) / (unsigned)d12;
    const unsigned m2 = ((1u << 20) + (unsigned)dim[2] - 1u) / (unsigned)dim[2];
    for (int s = lane; s < (int)vol; s += 32) {
      const float2 b = box[s];
      if (b.x != 0.f || b.y != 0.f) {
        const int x = (int)(((unsigned)s * m12) >> 20);
        const int r = s - x * d12;
        const int y = (int)(((unsigned)r * m2) >> 20);
        const int z = r - y * dim[2];
        const int64_t l = (int64_t)(lo[0] + x) * nn + (int64_t)(lo[1] + y) * N + (lo[2] + z);
        if (b.x != 0.f) atomicAdd(g_num + l, (double)b.x);
        if (b.y != 0.f) atomicAdd(g_den + l, (double)b.y);
        box[s] = make_float2(0.f, 0.f);
      }
    }
    __syncwarp();  // slots cleared before the next group's steps
  }
  // duplicate columns carrying counts above 256 (w = kDupMark) share their
  // pixel's geometry and add numerator only
  for (int64_t i = g.n_pix + threadIdx.x; i < g.ld_pix; i += kAggThreads) {
    const int4 qi = g.qi[i];
    if (qi.w == 0) continue;
    int f[3];
    float t[3];
    const float4 qhf = make_float4((float)qi.x * 0x1p-12f, (float)qi.y * 0x1p-12f,
                                   (float)qi.z * 0x1p-12f, 0.f);
    rotate_fx(Rh, Rhf, Rl, qi, qhf, g.qlo[i], N, f, t);
    reduce_direct<INTERIOR>(f, t, Nr[i] * inv_d, qi.w == 1 ? dv : 0.f, N, g_num, g_den);
  }
}

cudaError_t launch_compress(const Geom& g, const RotFX* rot, int64_t nrot, const float* Num,
                            const float* den, int mode, double* g_num, double* g_den, int nrep,
                            cudaStream_t s) {
  if (nrot <= 0) return cudaSuccess;
  const int64_t n_vox = (int64_t)g.N * g.N * g.N;
  if (g.interior)
    compress_kernel<true><<<(unsigned)nrot, kAggThreads, kAggSmem, s>>>(
        g, rot, Num, den, mode, g_num, g_den, nrep, n_vox);
  else
    compress_kernel<false><<<(unsigned)nrot, kAggThreads, kAggSmem, s>>>(
        g, rot, Num, den, mode, g_num, g_den, nrep, n_vox);
  return cudaGetLastError();
}

}  // namespace emc
