// emc_common.cuh -- device helpers shared by the libemc kernels (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/emc.h"

namespace emc {

// ---------------------------------------------------------------------------
// Device status word: the first error recorded wins.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Double-float ("f2") arithmetic: value = h + l with |l| <= ulp(h)/2.
// Rotated pixel coordinates need ~1e-8 voxel accuracy (the scores of Eq. 2.3
// react to log W at the 1e-7 level), which plain FP32 (ulp(64) = 7.6e-6)
// cannot give; FP64 is rare on this part, so pairs of FP32 are used instead.
// ---------------------------------------------------------------------------
struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ f2 two_prod(float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  f2 p = two_prod(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  return fast_two_sum(p.h, p.l);
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
  f2 s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}

// Rotation R (row-major 3x3) as double-float pairs.
struct RotDF {
  f2 r[9];
};

// Hamilton rotation matrix of a unit quaternion (w, x, y, z), in FP64.
__host__ __device__ __forceinline__ void quat_to_rot(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// The same, split into double-float pairs.
__host__ __device__ __forceinline__ void quat_to_rot_df(const double* q, RotDF* out) {
  double R[9];
  quat_to_rot(q, R);
  for (int t = 0; t < 9; t++) {
    float h = (float)R[t];
    out->r[t].h = h;
    out->r[t].l = (float)(R[t] - (double)h);
  }
}

// Grid coordinate p = R q + N/2 of one pixel, split into the integer corner
// f (floor) and the fraction t in [0, 1], both accurate to ~1e-9 voxel.
// Compensated dot product: with R = Rh + Rl and q = qh + ql,
//   p = N/2 + sum_b Rh_b qh_b + sum_b (Rh_b ql_b + Rl_b qh_b) + O(2^-40),
// the products Rh_b qh_b are split exactly (FMA), summed onto N/2 with exact
// two-sums, and every remainder is gathered in one small FP32 term.
__device__ __forceinline__ void rotate_to_grid(const RotDF& R, float4 qh, float4 ql, float half_n,
                                               int* f, float* t) {
  const float qhv[3] = {qh.x, qh.y, qh.z}, qlv[3] = {ql.x, ql.y, ql.z};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float S = half_n, L = 0.f;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const f2 r = R.r[3 * a + b];
      const f2 p = two_prod(r.h, qhv[b]);
      const f2 s = two_sum(S, p.h);
      S = s.h;
      L += s.l + fmaf(r.h, qlv[b], fmaf(r.l, qhv[b], p.l));
    }
    float fl = floorf(S);
    float fr = (S - fl) + L;  // S - fl is exact
    if (fr < 0.f) {
      fl -= 1.f;
      fr += 1.f;
    } else if (fr >= 1.f) {
      fl += 1.f;
      fr -= 1.f;
    }
    f[a] = (int)fl;
    t[a] = fminf(fmaxf(fr, 0.f), 1.f);
  }
}

// The same grid point in fixed point. With q = qi 2^-12 + qlo (qi integer,
// |qlo| <= 2^-13) and R = Rh 2^-20 + Rl (Rh integer, |Rl| <= 2^-21),
//   p = N/2 + sum_b Rh_b qi_b 2^-32 + sum_b (Rh_b 2^-20 qlo_b + Rl_b qi_b 2^-12)
// up to |Rl qlo| < 2^-34: the first sum is exact in 64-bit integers (its high
// word the floor, its low word the fraction to 2^-32), the small terms
// (|.| < 1e-3) take six FP32 FMAs. Rhf = Rh 2^-20 and qhf = qi 2^-12 as FP32
// (exact). Same accuracy as rotate_to_grid at a third of its instructions.
__device__ __forceinline__ void rotate_fx(const int* Rh, const float* Rhf, const float* Rl,
                                          int4 qi, float4 qhf, float4 qlo, int N, int* f,
                                          float* t) {
  const int qiv[3] = {qi.x, qi.y, qi.z};
  const float qhv[3] = {qhf.x, qhf.y, qhf.z}, qlv[3] = {qlo.x, qlo.y, qlo.z};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    long long acc = ((long long)(N >> 1) << 32) + ((N & 1) ? (1LL << 31) : 0LL);
#pragma unroll
    for (int b = 0; b < 3; b++) acc += (long long)Rh[3 * a + b] * (long long)qiv[b];
    const float small =
        fmaf(Rhf[3 * a], qlv[0],
             fmaf(Rhf[3 * a + 1], qlv[1],
                  fmaf(Rhf[3 * a + 2], qlv[2],
                       fmaf(Rl[3 * a], qhv[0], fmaf(Rl[3 * a + 1], qhv[1], Rl[3 * a + 2] * qhv[2])))));
    int fl = (int)(acc >> 32);
    // the 32-bit fraction as FP32 without a conversion instruction: its top 23
    // bits as the mantissa of a number in [1, 2), the low 9 bits likewise
    const unsigned fw = (unsigned)(acc & 0xffffffffLL);
    const float fhi = __uint_as_float(0x3f800000u | (fw >> 9)) - 1.0f;           // exact
    const float flo = __uint_as_float(0x3f800000u | ((fw & 511u) << 14)) - 1.0f;  // exact
    float fr = fhi + fmaf(flo, 0x1p-23f, small);
    if (fr < 0.f) {
      fl -= 1;
      fr += 1.f;
    } else if (fr >= 1.f) {
      fl += 1;
      fr -= 1.f;
    }
    f[a] = fl;
    t[a] = fminf(fmaxf(fr, 0.f), 1.f);
  }
}

// Trilinear value (Eq. 2.8, tent weights) at p = f + t from the grid in its
// corner-pair layout g4[(x N + y) N + z] = (g[x][y][z], g[x][y][z+1],
// g[x][y+1][z], g[x][y+1][z+1]) (0 beyond the grid): two 16-byte loads per
// point where the plain layout needs eight scattered 4-byte ones, which is
// what limits the expansion (its loads are gathers: every lane of a warp reads
// another cache line). Corners inside the grid only (interior points).
__device__ __forceinline__ float trilinear_g4(const float4* __restrict__ g4, int N, const int* f,
                                              const float* t) {
  const int64_t o = ((int64_t)f[0] * N + f[1]) * N + f[2];
  const float4 a = __ldg(g4 + o), b = __ldg(g4 + o + (int64_t)N * N);
  const float tz = t[2], sz = 1.f - tz, ty = t[1], sy = 1.f - ty;
  const float va = sy * fmaf(tz, a.y, sz * a.x) + ty * fmaf(tz, a.w, sz * a.z);
  const float vb = sy * fmaf(tz, b.y, sz * b.x) + ty * fmaf(tz, b.w, sz * b.z);
  return fmaf(t[0], vb, (1.f - t[0]) * va);
}

// FP32 -> FP64 with integer operations (the conversion instruction runs on the
// FP64 pipe, at 1/64 of the FP32 rate on this part): sign, exponent rebiased by
// 1023 - 127, mantissa moved up 29 bits; a subnormal input a 2^-149 is
// normalised by its leading bit. Exact for every finite input.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t a = u & 0x7fffffffu;
  const unsigned long long sgn = ((unsigned long long)(u >> 31)) << 63;
  unsigned long long d;
  if (a >= 0x00800000u) {
    d = ((unsigned long long)a + (896ull << 23)) << 29;
  } else if (a != 0u) {
    const int p = 31 - __clz(a);  // a = 2^p (1 + f), p < 23
    d = ((unsigned long long)(p - 149 + 1023) << 52) |
        (((unsigned long long)a << (52 - p)) & 0xfffffffffffffull);
  } else {
    d = 0ull;
  }
  return __longlong_as_double((long long)(sgn | d));
}

// ---------------------------------------------------------------------------
// BF16 helpers (round to nearest even).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ float bf16_val(uint16_t u) {
  return __uint_as_float(((uint32_t)u) << 16);
}

// FP16 helpers (round to nearest even).
__device__ __forceinline__ uint16_t fp16_bits(float x) {
  __half h = __float2half_rn(x);
  return *reinterpret_cast<uint16_t*>(&h);
}
__device__ __forceinline__ float fp16_val(uint16_t u) {
  return __half2float(*reinterpret_cast<const __half*>(&u));
}

// The fixed grid of the hi term of the BF16 three-term split: multiples of
// 1/8 in [-32, 32); every such value has at most 8 significant bits (exact in
// BF16) and sums of (integer count <= 256) x (hi) stay on the 1/8 grid, so
// FP32 accumulates them exactly while |sum| < 2^21.
constexpr float kHiScale = 8.0f;
constexpr float kHiMin = -32.0f;
constexpr float kHiMax = 32.0f - 0.125f;
// The FP16 two-term split: hi on the 1/64 grid in [-32, 32) (at most 11
// significant bits, exact in FP16); counts <= 2048 are exact in FP16 and the
// products and partial sums stay on the 1/64 grid, exact in FP32 while
// |sum| < 2^18.
constexpr float kHi16Scale = 64.0f;
constexpr float kHi16Max = 32.0f - 1.0f / 64.0f;
// Scores are split for the epilogues into a part on the 1/64 grid (every
// 1/8-grid value lies on it) and a small rest; references (maxima, lse) use
// the same grid so that subtracting them is exact.
constexpr float kGrid = 64.0f;
constexpr double kGridD = 64.0;
// FP16 responsibilities are stored scaled by 2^14 (P <= 1 stays below the
// FP16 maximum, P down to ~4e-9 stays normal); the update removes the scale.
constexpr float kP16Scale = 16384.0f;

// Duplicate pixel columns for counts above 256 (EMC_FLAG_WIDE_COUNTS): at most
// this many, each carrying up to kDupCount photons of its source pixel; their
// geometry entry has w = kDupMark (used pixels 1, padding 0).
constexpr int kDupCols = 64;
constexpr int kDupCount = 256;
constexpr float kDupMark = 2.0f;

// Gaussian model (Eqs. 2.2-2.3): S_jk <= log w_j < 0, and scores further than
// kGaussClamp below zero are clamped -- their exp vanishes next to any
// frame's best rotation, and the clamp keeps every score's 1/64-grid part
// exact in FP32.
constexpr float kGaussClamp = 120000.0f;

// Scale of the Gaussian contraction, from the grid maximum Wmax and the
// largest frame total Nmax (x: s, y: 1/s^2):
//   s  = the largest power of two with s Wmax Nmax <= 2^23 and s Wmax <= 2^15.
//        The integral hi part of s W is at most s Wmax + 1/2, so every partial
//        sum of hi K over a frame stays below 2^24 (exact in FP32) and hi
//        stays far inside the FP16 range.
__host__ __device__ inline float4 gauss_scales(float wmax, long long nmax) {
  if (!(wmax > 0.f) || !(wmax < 3.0e38f)) return make_float4(1.f, 1.f, 0.f, 0.f);
  const double w = (double)wmax, n = (double)(nmax > 0 ? nmax : 1);
  int e = ilogb(8388608.0 / (w * n));
  const int e2 = ilogb(32768.0 / w);
  e = e < e2 ? e : e2;
  e = e < -60 ? -60 : (e > 60 ? 60 : e);
  return make_float4((float)ldexp(1.0, e), (float)ldexp(1.0, -2 * e), 0.f, 0.f);
}

}  // namespace emc
