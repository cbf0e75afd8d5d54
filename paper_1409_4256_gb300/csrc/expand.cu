// expand.cu -- e-step of EMC (Eq. 2.9) and the per-rotation bias of Eq. 2.3.
//
// One CTA per rotation row j, threads striding over pixels. For every pixel
// the grid point p = R_j q_i + N/2 is formed in double-float (R_j from the
// context's table of double-float rotation matrices), the trilinear
// weights f(p_l - p) of the eight surrounding voxels (Eq. 2.8, tent kernel)
// blend the L2-resident grid, W_ij = max(W, w_floor) and log W_ij is stored in
// the layout the contraction of the chosen precision reads. The same CTA sums
// W_ij over pixels in FP64 (block reduction) and writes
//   bias_j = log w_j - sum_i W_ij,
// the rotation-only part of S_jk = sum_i K_ik log W_ij - W_ij + log w_j
// (per-thread compensated FP32 sums, FP64 across the block).
// Writes are coalesced along pixels; HBM traffic is the L write (4 B/(i,j)
// for FP32, 2 B for BF16, 6 B for the three-term split, 4 B for the FP16 split).
//
// Gaussian model (GAUSS): no floor and no logarithm. s W_ij (s = 2^e from the
// context's scales) is split into three FP16 terms: hi integral (rint below
// 2048, else the FP16 rounding, itself integral there), mid = fp16(s W - hi),
// lo = fp16(s W - hi - mid); the representation error is below 2^-23 s^-1 W
// units. The CTA sums W_ij^2 instead, bias_j = log w_j - sum_i W_ij^2 / (2 sigma^2).
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

constexpr int kExpandThreads = 256;

// Trilinear value of the grid at p = f + t (Eq. 2.8 tent weights). INTERIOR:
// all eight corners are known to lie inside the grid (no bounds checks, one
// base index); otherwise corners outside [0, N) carry no value.
template <bool INTERIOR>
__device__ __forceinline__ float trilinear(const float* __restrict__ grid, int N, const int* f,
                                           const float* t) {
  const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
  float W = 0.f;
  if (INTERIOR) {
    const int nn = N * N;
    const float* g = grid + (f[0] * nn + f[1] * N + f[2]);
#pragma unroll
    for (int cx = 0; cx < 2; cx++)
#pragma unroll
      for (int cy = 0; cy < 2; cy++) {
        const float wxy = wx[cx] * wy[cy];
        const float* gr = g + cx * nn + cy * N;
        W = fmaf(wxy * wz[0], __ldg(gr), W);
        W = fmaf(wxy * wz[1], __ldg(gr + 1), W);
      }
    return W;
  }
  const int64_t nn = (int64_t)N * N;
#pragma unroll
  for (int c = 0; c < 8; c++) {
    int x = f[0] + ((c >> 2) & 1), y = f[1] + ((c >> 1) & 1), z = f[2] + (c & 1);
    if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= N) continue;
    const float w = wx[(c >> 2) & 1] * wy[(c >> 1) & 1] * wz[c & 1];
    W = fmaf(w, __ldg(grid + (int64_t)x * nn + (int64_t)y * N + z), W);
  }
  return W;
}

template <int PREC, bool GAUSS, bool INTERIOR>
__global__ void __launch_bounds__(kExpandThreads)
    expand_kernel(const float4* __restrict__ qh, const float4* __restrict__ ql, int64_t n_pix,
                  int64_t ld_pix, int N, const float* __restrict__ grid,
                  const float4* __restrict__ g4,
                  const RotDF* __restrict__ rot, const double* __restrict__ logw, int64_t nrot,
                  float w_floor, void* __restrict__ Lbase, int64_t plane_stride,
                  double* __restrict__ bias, const float4* __restrict__ gsc, double inv2s2,
                  int32_t* status) {
  const int64_t row = blockIdx.x;
  __shared__ RotDF R;
  __shared__ double red[kExpandThreads / 32];
  const bool valid_row = row < nrot;
  if (threadIdx.x < 18 && valid_row)
    reinterpret_cast<float*>(&R)[threadIdx.x] = reinterpret_cast<const float*>(rot + row)[threadIdx.x];
  __syncthreads();

  float* Lf = reinterpret_cast<float*>(Lbase) + row * ld_pix;
  uint16_t* Lb = reinterpret_cast<uint16_t*>(Lbase) + row * ld_pix;
  const float half_n = 0.5f * (float)N;
  float wsum = 0.f, wcomp = 0.f;  // Kahan-compensated sum of W (W^2) over this thread's pixels
  int bad = 0, nonfinite = 0;
  const float gs = GAUSS ? gsc->x : 1.f;

  for (int64_t i = threadIdx.x; i < ld_pix; i += kExpandThreads) {
    float L = 0.f;
    bool used = false;
    if (valid_row) {  // geometry w: 1 pixel, kDupMark duplicate column, 0 padding / ones
      float4 a = qh[i], b = ql[i];
      if (a.w != 0.f) {
        used = true;
        int f[3];
        float t[3];
        rotate_to_grid(R, a, b, half_n, f, t);
        float W = (INTERIOR && g4) ? trilinear_g4(g4, N, f, t) : trilinear<INTERIOR>(grid, N, f, t);
        nonfinite |= !(fabsf(W) <= 3.4e38f);  // a NaN or infinite voxel of the model
        W = fmaxf(W, GAUSS ? 0.f : w_floor);
        if (a.w == 1.f) {  // duplicate columns (counts above 256) repeat a pixel: not summed
          const float ky = (GAUSS ? W * W : W) - wcomp;
          const float kt = wsum + ky;
          wcomp = (kt - wsum) - ky;
          wsum = kt;
        }
        L = GAUSS ? W * gs : logf(W);
      }
    }
    if (GAUSS) {
      const float hi = L < 2048.f ? rintf(L) : fp16_val(fp16_bits(L));
      const float r = L - hi;  // exact
      const uint16_t mid = fp16_bits(r);
      Lb[i] = fp16_bits(hi);
      Lb[i + plane_stride] = mid;
      Lb[i + 2 * plane_stride] = fp16_bits(r - fp16_val(mid));
    } else if (PREC == EMC_PREC_FP32) {
      Lf[i] = L;
    } else if (PREC == EMC_PREC_BF16) {
      Lb[i] = bf16_bits(L);
    } else if (PREC == EMC_PREC_FP16_SPLIT) {
      // two-term FP16 split: hi on the 1/64 grid, rest r (|r| <= 1/128)
      float hi = rintf(L * kHi16Scale) * (1.0f / kHi16Scale);
      if (used && (hi < kHiMin || hi > kHi16Max)) bad = 1;
      hi = fminf(fmaxf(hi, kHiMin), kHi16Max);
      Lb[i] = fp16_bits(hi);
      Lb[i + plane_stride] = fp16_bits(L - hi);
    } else {
      // three-term split: hi on the 1/8 grid, residual r = mid + lo
      float hi = rintf(L * kHiScale) * (1.0f / kHiScale);
      if (used && (hi < kHiMin || hi > kHiMax)) bad = 1;
      hi = fminf(fmaxf(hi, kHiMin), kHiMax);
      float r = L - hi;  // exact
      uint16_t mid = bf16_bits(r);
      uint16_t lo = bf16_bits(r - bf16_val(mid));
      Lb[i] = bf16_bits(hi);
      Lb[i + plane_stride] = mid;
      Lb[i + 2 * plane_stride] = lo;
    }
  }
  if (nonfinite) set_status(status, EMC_ERR_NUMERIC);
  if (bad) set_status(status, EMC_ERR_UNSUPPORTED);

  // FP64 block reduction of sum_i W_ij
  double ws = (double)wsum - (double)wcomp;
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kExpandThreads / 32; w++) s += red[w];
    bias[row] = valid_row ? logw[row] - (GAUSS ? s * inv2s2 : s) : -INFINITY;
  }
}

// Poisson-fluence model: L_ij = log(W_ij / B_j) + c with B_j = sum_i W_ij,
// so that sum_i K_ik L_ij = sum_i K_ik log W_ij - N_k log B_j + c N_k, the
// scores of the maximum-likelihood fluence phi_jk = N_k / B_j up to the
// per-frame shift c N_k (removed in FP64 by the log-sum-exp merge). B_j is
// needed before the first L is written, so the CTA runs two phases: W_ij
// (stashed in shared memory when the row fits, STASH, else interpolated again)
// and its sum, then the split of log W_ij + a_j, a_j = c - log B_j. a_j is
// carried as ah (1/8 grid) + al: x + ah is formed with its exact rounding
// error e (two-sum), hi is the 1/8-grid rounding of the whole x + ah + e + al,
// and the rest r = ((x + ah - hi) + e) + al goes to mid + lo. No per-rotation
// rounding of a_j enters the contraction (it would be multiplied by N_k), and
// the rest stays centred on zero: were al left in every rest, the mid/lo
// accumulator would grow to N_k al and round at that size on every K step.
// bias = double[2][rows]: log w_j, then B_j
// (FP64); Bctx[row] = B_j as well (the context's copy for the sparse steps).
template <bool INTERIOR, bool STASH>
__global__ void __launch_bounds__(kExpandThreads)
    expand_flu_kernel(const float4* __restrict__ qh, const float4* __restrict__ ql,
                      int64_t ld_pix, int N, const float* __restrict__ grid,
                      const float4* __restrict__ g4,
                      const RotDF* __restrict__ rot, const double* __restrict__ logw, int64_t nrot,
                      float w_floor, double c, uint16_t* __restrict__ Lbase, int64_t plane_stride,
                      double* __restrict__ bias, double* __restrict__ Bctx, int32_t* status) {
  extern __shared__ float wst[];  // STASH: W of the row's pixels
  const int64_t row = blockIdx.x;
  __shared__ RotDF R;
  __shared__ double red[kExpandThreads / 32];
  __shared__ float a_split[2];
  const bool valid_row = row < nrot;
  if (threadIdx.x < 18 && valid_row)
    reinterpret_cast<float*>(&R)[threadIdx.x] = reinterpret_cast<const float*>(rot + row)[threadIdx.x];
  __syncthreads();
  const float half_n = 0.5f * (float)N;
  float wsum = 0.f, wcomp = 0.f;
  int nonfinite = 0;
  if (valid_row) {
    for (int64_t i = threadIdx.x; i < ld_pix; i += kExpandThreads) {
      const float4 a = qh[i];
      if (a.w == 0.f) continue;
      int f[3];
      float t[3];
      rotate_to_grid(R, a, ql[i], half_n, f, t);
      const float Wt = (INTERIOR && g4) ? trilinear_g4(g4, N, f, t)
                                        : trilinear<INTERIOR>(grid, N, f, t);
      nonfinite |= !(fabsf(Wt) <= 3.4e38f);  // a NaN or infinite voxel of the model
      const float W = fmaxf(Wt, w_floor);
      if (STASH) wst[i] = W;
      if (a.w == 1.f) {  // duplicate columns repeat a pixel: not summed
        const float ky = W - wcomp;
        const float kt = wsum + ky;
        wcomp = (kt - wsum) - ky;
        wsum = kt;
      }
    }
  }
  if (nonfinite) set_status(status, EMC_ERR_NUMERIC);
  double ws = (double)wsum - (double)wcomp;
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double B = 0.0;
    for (int w = 0; w < kExpandThreads / 32; w++) B += red[w];
    const double aj = valid_row ? c - log(B) : 0.0;
    const float ah = (float)(rint(aj * kHiScale) / kHiScale);
    a_split[0] = ah;
    a_split[1] = (float)(aj - (double)ah);
    bias[row] = valid_row ? logw[row] : -INFINITY;
    bias[gridDim.x + row] = valid_row ? B : 0.0;
    Bctx[row] = valid_row ? B : 0.0;
  }
  __syncthreads();
  const float ah = a_split[0], al = a_split[1];
  uint16_t* Lb = Lbase + row * ld_pix;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < ld_pix; i += kExpandThreads) {
    float hi = 0.f, r = 0.f;
    const float4 a = qh[i];
    if (valid_row && a.w != 0.f) {
      float W;
      if (STASH) {
        W = wst[i];
      } else {
        int f[3];
        float t[3];
        rotate_to_grid(R, a, ql[i], half_n, f, t);
        W = fmaxf((INTERIOR && g4) ? trilinear_g4(g4, N, f, t) : trilinear<INTERIOR>(grid, N, f, t),
                  w_floor);
      }
      const float x = logf(W);
      const float s = x + ah;  // two-sum: s + e = x + ah exactly
      const float bb = s - x;
      const float e = (x - (s - bb)) + (ah - bb);
      hi = rintf((s + (e + al)) * kHiScale) * (1.0f / kHiScale);
      if (hi < kHiMin || hi > kHiMax) bad = 1;
      hi = fminf(fmaxf(hi, kHiMin), kHiMax);
      r = ((s - hi) + e) + al;
    }
    const uint16_t mid = bf16_bits(r);
    Lb[i] = bf16_bits(hi);
    Lb[i + plane_stride] = mid;
    Lb[i + 2 * plane_stride] = bf16_bits(r - bf16_val(mid));
  }
  if (bad) set_status(status, EMC_ERR_UNSUPPORTED);
}

// shared memory for one stashed row of W: rows up to 96 KB (24576 pixels)
constexpr size_t kFluStashMax = 96 * 1024;

cudaError_t launch_expand_flu(const Geom& g, const float* grid, const float4* g4, const RotDF* rot,
                              const double* logw, int64_t nrot, int64_t rows, int precision,
                              float w_floor, double c, Planes L, double* bias, double* Bctx,
                              int32_t* status, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (precision != EMC_PREC_BF16_SPLIT) return cudaErrorInvalidValue;
  const size_t stash = sizeof(float) * (size_t)g.ld_pix;
  const bool use_stash = stash <= kFluStashMax;
  dim3 grd((unsigned)rows), blk(kExpandThreads);
  cudaError_t e = cudaSuccess;
#define EMC_FLU(I, S)                                                                         \
  do {                                                                                        \
    const size_t sm = S ? stash : 0;                                                          \
    if (sm > 48 * 1024)                                                                       \
      e = cudaFuncSetAttribute(expand_flu_kernel<I, S>,                                       \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);         \
    if (e == cudaSuccess)                                                                     \
      expand_flu_kernel<I, S><<<grd, blk, sm, s>>>(                                           \
          g.qh, g.ql, g.ld_pix, g.N, grid, g4, rot, logw, nrot, w_floor, c,                   \
          reinterpret_cast<uint16_t*>(L.base), L.plane_stride, bias, Bctx, status);           \
  } while (0)
  if (g.interior) {
    if (use_stash) EMC_FLU(true, true);
    else EMC_FLU(true, false);
  } else {
    if (use_stash) EMC_FLU(false, true);
    else EMC_FLU(false, false);
  }
#undef EMC_FLU
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_expand(const Geom& g, const float* grid, const float4* g4, const RotDF* rot,
                          const double* logw, int64_t nrot, int64_t rows, int precision,
                          float w_floor, Planes L, double* bias, const float4* gsc, double sigma,
                          int32_t* status, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  dim3 grd((unsigned)rows), blk(kExpandThreads);
#define EMC_EXPAND_I(P, G, I)                                                                \
  expand_kernel<P, G, I><<<grd, blk, 0, s>>>(g.qh, g.ql, g.n_pix, g.ld_pix, g.N, grid, g4, rot, \
                                             logw, nrot, w_floor, L.base, L.plane_stride, bias, \
                                             gsc, gsc ? 1.0 / (2.0 * sigma * sigma) : 0.0, status)
#define EMC_EXPAND(P, G)        \
  if (g.interior) {             \
    EMC_EXPAND_I(P, G, true);   \
  } else {                      \
    EMC_EXPAND_I(P, G, false);  \
  }
  if (gsc) {
    EMC_EXPAND(EMC_PREC_FP16_SPLIT, true);
  } else {
    switch (precision) {
      case EMC_PREC_FP32: EMC_EXPAND(EMC_PREC_FP32, false); break;
      case EMC_PREC_BF16: EMC_EXPAND(EMC_PREC_BF16, false); break;
      case EMC_PREC_FP16_SPLIT: EMC_EXPAND(EMC_PREC_FP16_SPLIT, false); break;
      default: EMC_EXPAND(EMC_PREC_BF16_SPLIT, false); break;
    }
  }
#undef EMC_EXPAND
#undef EMC_EXPAND_I
  return cudaGetLastError();
}

}  // namespace emc
