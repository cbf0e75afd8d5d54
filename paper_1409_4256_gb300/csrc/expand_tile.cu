// expand_tile.cu -- e-step of EMC (Eq. 2.9) for the Poisson model, one row
// tile of 128 rotations per CTA (and a slice of 256 pixels: small CTAs, so
// that the last wave of the grid leaves few SMs idle).
//
// Each thread owns two neighbouring pixels and takes the tile's rotations in
// turn, so the pixels' geometry stays in registers and the rotations come from
// shared memory. Per (i, j): the grid point p = R_j q_i + N/2, the trilinear
// value of the model (Eq. 2.8, tent weights), W_ij = max(W, w_floor) and
// log W_ij in the layout of the chosen precision (as expand.cu), written two
// pixels at a time. The row sums sum_i W_ij of the bias
//   bias_j = log w_j - sum_i W_ij
// are kept as double-float pairs of FP32 (exact two-sums: FP64 is rare on
// this part, and a per-row FP64 reduction kept its pipe 65% busy). A warp
// parks its lanes' pairs of eight rows in shared memory and reduces them
// transposed (each lane sums a quarter of one row, two shuffles finish it),
// a quarter of the instructions of eight butterfly reductions; the CTA adds
// its warps' sums, and a second kernel the slices' partial sums in slice
// order (deterministic).
//
// The grid point is formed in fixed point (rotate_fx): exact 64-bit integer
// products for the large part, six FP32 FMAs for the rest (error ~1e-10
// voxel), where expand.cu uses double-float arithmetic.
//
// With the last iteration's L (DELTA), the CTA also reads the previous planes
// of its elements and keeps, per pixel, the largest rise and fall of the
// represented log W over the tile's rows: the rows t and ntp + t of the
// incremental bound's increments D (prune.cu), rounded up to the operand type
// of the frames, and their magnitude bound A (the rows 2 ntp + t).
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

namespace {

constexpr int kTThreads = 128;
constexpr int kTRows = 128;
constexpr int kTPix = 2 * kTThreads;

// one rotation in shared memory: read as seven 16-byte words
struct __align__(16) RowFX {
  int hi[9];
  float hf[9];  // hi as FP32 (hi 2^-20, exact)
  float lo[9];
  float pad;
};

template <bool INTERIOR>
__device__ __forceinline__ float trilinear_fx(const float* __restrict__ grid, int N, const int* f,
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
    const int x = f[0] + ((c >> 2) & 1), y = f[1] + ((c >> 1) & 1), z = f[2] + (c & 1);
    if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= N) continue;
    W = fmaf(wx[(c >> 2) & 1] * wy[(c >> 1) & 1] * wz[c & 1],
             __ldg(grid + (int64_t)x * nn + (int64_t)y * N + z), W);
  }
  return W;
}

// value of one element of L in the precision's layout (old planes, DELTA)
template <int PREC>
__device__ __forceinline__ float2 read_pair(const void* L, int64_t o, int64_t ps) {
  if (PREC == EMC_PREC_FP32) return *reinterpret_cast<const float2*>((const float*)L + o);
  const uint16_t* b = (const uint16_t*)L;
  auto val = [&](int64_t oo) -> float2 {
    const uint32_t u = *reinterpret_cast<const uint32_t*>(b + oo);
    if (PREC == EMC_PREC_FP16_SPLIT)
      return make_float2(fp16_val((uint16_t)(u & 0xffffu)), fp16_val((uint16_t)(u >> 16)));
    return make_float2(bf16_val((uint16_t)(u & 0xffffu)), bf16_val((uint16_t)(u >> 16)));
  };
  float2 v = val(o);
  const int np = PREC == EMC_PREC_BF16_SPLIT ? 3 : (PREC == EMC_PREC_FP16_SPLIT ? 2 : 1);
  for (int q = 1; q < np; q++) {
    const float2 w = val(o + q * ps);
    v.x += w.x;  // planes of one element: their sum rounds at most twice
    v.y += w.y;
  }
  return v;
}

template <int PREC>
__device__ __forceinline__ uint16_t round_up_operand(float x) {
  if (PREC == EMC_PREC_FP16_SPLIT) {
    __half h = __float2half_ru(x);
    return *reinterpret_cast<uint16_t*>(&h);
  }
  __nv_bfloat16 b = __float2bfloat16_ru(x);
  return *reinterpret_cast<uint16_t*>(&b);
}

template <int PREC, bool INTERIOR, bool DELTA>
__global__ void __launch_bounds__(kTThreads, 6)
    expand_tile_kernel(const int4* __restrict__ qi_g, const float4* __restrict__ qlo_g,
                       int64_t ld_pix, int N, const float* __restrict__ grid,
                       const float4* __restrict__ g4,
                       const RotFX* __restrict__ rot, int64_t nrot, int64_t rows, float w_floor,
                       void* __restrict__ Lbase, int64_t ps, double* __restrict__ partial,
                       const void* __restrict__ Lold, uint16_t* __restrict__ D, int64_t ntp,
                       int32_t* status) {
  __shared__ RowFX R[kTRows];
  __shared__ float2 rsum[kTThreads / 32][kTRows];
  // eight rows of every lane's pair, rows padded to 33 so that the transposed
  // reads hit 16 distinct bank pairs per half warp
  __shared__ float2 park[kTThreads / 32][8 * 33];
  const int64_t t = blockIdx.y;
  const int64_t r0 = t * kTRows;
  const int nr = (int)min((int64_t)kTRows, nrot - r0);  // >= 1 for every tile of rows
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int x = threadIdx.x; x < kTRows * 9; x += kTThreads) {
    const int r = x / 9, e = x % 9;
    int h = 0;
    float l = 0.f;
    if (r < nr) {
      h = rot[r0 + r].hi[e];
      l = rot[r0 + r].lo[e];
    }
    R[r].hi[e] = h;
    R[r].hf[e] = (float)h * 0x1p-20f;
    R[r].lo[e] = l;
  }
  const int64_t i0 = (int64_t)blockIdx.x * kTPix + 2 * threadIdx.x;
  const bool inside = i0 < ld_pix;  // ld_pix is even: both pixels or neither
  int4 qi[2];
  float4 qh[2], ql[2];
#pragma unroll
  for (int u = 0; u < 2; u++) {
    qi[u] = inside ? qi_g[i0 + u] : make_int4(0, 0, 0, 0);
    ql[u] = inside ? qlo_g[i0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
    qh[u] = make_float4((float)qi[u].x * 0x1p-12f, (float)qi[u].y * 0x1p-12f,
                        (float)qi[u].z * 0x1p-12f, 0.f);
  }
  __syncthreads();
  float dp[2] = {-INFINITY, -INFINITY}, dm[2] = {-INFINITY, -INFINITY};
  int bad = 0, nonfinite = 0;
  for (int r = 0; r < kTRows; r++) {
    const int64_t row = r0 + r;
    const bool vrow = r < nr;
    float L[2] = {0.f, 0.f};
    float s = 0.f, se = 0.f;  // row sum of the pair as s + se
    const RowFX Rr = R[r];
#pragma unroll
    for (int u = 0; u < 2; u++) {
      if (vrow && qi[u].w != 0) {  // w: 1 pixel, 2 duplicate column, 0 padding / ones
        int f[3];
        float tt[3];
        rotate_fx(Rr.hi, Rr.hf, Rr.lo, qi[u], qh[u], ql[u], N, f, tt);
        float W = (INTERIOR && g4) ? trilinear_g4(g4, N, f, tt)
                                   : trilinear_fx<INTERIOR>(grid, N, f, tt);
        nonfinite |= !(fabsf(W) <= 3.4e38f);  // a NaN or infinite voxel of the model
        W = fmaxf(W, w_floor);
        if (qi[u].w == 1) {  // duplicate columns repeat a pixel: not summed
          const f2 a = two_sum(s, W);
          s = a.h;
          se += a.l;
        }
        L[u] = logf(W);
      }
    }
    if (inside && row < rows) {
      const int64_t o = row * ld_pix + i0;
      // DELTA: the change of the represented value (the planes' sum) of each element
      if (PREC == EMC_PREC_FP32) {
        *reinterpret_cast<float2*>((float*)Lbase + o) = make_float2(L[0], L[1]);
        if (DELTA && vrow) {
          const float2 old = read_pair<PREC>(Lold, o, ps);
          const float d0 = L[0] - old.x, d1 = L[1] - old.y;
          dp[0] = fmaxf(dp[0], d0); dm[0] = fmaxf(dm[0], -d0);
          dp[1] = fmaxf(dp[1], d1); dm[1] = fmaxf(dm[1], -d1);
        }
      } else if (PREC == EMC_PREC_BF16) {
        const uint16_t b0 = bf16_bits(L[0]), b1 = bf16_bits(L[1]);
        *reinterpret_cast<uint32_t*>((uint16_t*)Lbase + o) = (uint32_t)b0 | ((uint32_t)b1 << 16);
        if (DELTA && vrow) {
          const float2 old = read_pair<PREC>(Lold, o, ps);
          const float d0 = bf16_val(b0) - old.x, d1 = bf16_val(b1) - old.y;
          dp[0] = fmaxf(dp[0], d0); dm[0] = fmaxf(dm[0], -d0);
          dp[1] = fmaxf(dp[1], d1); dm[1] = fmaxf(dm[1], -d1);
        }
      } else if (PREC == EMC_PREC_FP16_SPLIT) {
        uint16_t h[2], rr[2];
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          float hi = rintf(L[u] * kHi16Scale) * (1.0f / kHi16Scale);
          if (vrow && qi[u].w != 0 && (hi < kHiMin || hi > kHi16Max)) bad = 1;
          hi = fminf(fmaxf(hi, kHiMin), kHi16Max);
          h[u] = fp16_bits(hi);
          rr[u] = fp16_bits(L[u] - hi);
          v[u] = hi + fp16_val(rr[u]);
        }
        uint16_t* Lb = (uint16_t*)Lbase + o;
        *reinterpret_cast<uint32_t*>(Lb) = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
        *reinterpret_cast<uint32_t*>(Lb + ps) = (uint32_t)rr[0] | ((uint32_t)rr[1] << 16);
        if (DELTA && vrow) {
          const float2 old = read_pair<PREC>(Lold, o, ps);
          const float d0 = v[0] - old.x, d1 = v[1] - old.y;
          dp[0] = fmaxf(dp[0], d0); dm[0] = fmaxf(dm[0], -d0);
          dp[1] = fmaxf(dp[1], d1); dm[1] = fmaxf(dm[1], -d1);
        }
      } else {
        // three-term split: hi on the 1/8 grid, residual r = mid + lo
        uint16_t h[2], m[2], l[2];
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          float hi = rintf(L[u] * kHiScale) * (1.0f / kHiScale);
          if (vrow && qi[u].w != 0 && (hi < kHiMin || hi > kHiMax)) bad = 1;
          hi = fminf(fmaxf(hi, kHiMin), kHiMax);
          const float r = L[u] - hi;  // exact
          m[u] = bf16_bits(r);
          l[u] = bf16_bits(r - bf16_val(m[u]));
          h[u] = bf16_bits(hi);
          v[u] = (hi + bf16_val(m[u])) + bf16_val(l[u]);
        }
        uint16_t* Lb = (uint16_t*)Lbase + o;
        *reinterpret_cast<uint32_t*>(Lb) = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
        *reinterpret_cast<uint32_t*>(Lb + ps) = (uint32_t)m[0] | ((uint32_t)m[1] << 16);
        *reinterpret_cast<uint32_t*>(Lb + 2 * ps) = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
        if (DELTA && vrow) {
          const float2 old = read_pair<PREC>(Lold, o, ps);
          const float d0 = v[0] - old.x, d1 = v[1] - old.y;
          dp[0] = fmaxf(dp[0], d0); dm[0] = fmaxf(dm[0], -d0);
          dp[1] = fmaxf(dp[1], d1); dm[1] = fmaxf(dm[1], -d1);
        }
      }
    }
    // row sums: park the pair; every eighth row, lane l sums eight lanes'
    // pairs of row l mod 8, and the lanes l, l ^ 8, l ^ 16, l ^ 24 combine
    float2* pk = park[warp];
    pk[(r & 7) * 33 + lane] = make_float2(s, se);
    if ((r & 7) == 7) {
      __syncwarp();
      const float2* src = pk + (lane & 7) * 33 + (lane >> 3) * 8;
      float a = 0.f, ae = 0.f;
#pragma unroll
      for (int m = 0; m < 8; m++) {
        const float2 v = src[m];
        const f2 z = two_sum(a, v.x);
        a = z.h;
        ae += v.y + z.l;
      }
#pragma unroll
      for (int off = 8; off <= 16; off <<= 1) {
        const float ao = __shfl_xor_sync(0xffffffffu, a, off);
        const float eo = __shfl_xor_sync(0xffffffffu, ae, off);
        const f2 z = two_sum(a, ao);
        a = z.h;
        ae += eo + z.l;
      }
      if (lane < 8) rsum[warp][r - 7 + lane] = make_float2(a, ae);
      __syncwarp();
    }
  }
  if (nonfinite) set_status(status, EMC_ERR_NUMERIC);
  if (bad) set_status(status, EMC_ERR_UNSUPPORTED);
  __syncthreads();
  if (threadIdx.x < kTRows) {
    float s = 0.f, se = 0.f;
    if ((int)threadIdx.x < nr)
      for (int w = 0; w < kTThreads / 32; w++) {
        const float2 v = rsum[w][threadIdx.x];
        const f2 a = two_sum(s, v.x);
        s = a.h;
        se += v.y + a.l;
      }
    partial[(int64_t)blockIdx.x * rows + r0 + threadIdx.x] = f32_to_f64(s) + f32_to_f64(se);
  }
  if (DELTA && inside) {
    float a[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
      // the sum of the planes rounded at most twice: 2^-23 |d| covers it
      dp[u] += 2.0f * 1.1920929e-7f * fabsf(dp[u]);
      dm[u] += 2.0f * 1.1920929e-7f * fabsf(dm[u]);
      // bound of both rounded magnitudes (BF16 rounding up: at most 2^-7 relative)
      a[u] = fmaxf(fabsf(dp[u]), fabsf(dm[u])) * 1.0078125f;
    }
    const uint16_t p0 = round_up_operand<PREC>(dp[0]), p1 = round_up_operand<PREC>(dp[1]);
    const uint16_t m0 = round_up_operand<PREC>(dm[0]), m1 = round_up_operand<PREC>(dm[1]);
    const uint16_t a0 = round_up_operand<PREC>(a[0]), a1 = round_up_operand<PREC>(a[1]);
    *reinterpret_cast<uint32_t*>(D + t * ld_pix + i0) = (uint32_t)p0 | ((uint32_t)p1 << 16);
    *reinterpret_cast<uint32_t*>(D + (ntp + t) * ld_pix + i0) = (uint32_t)m0 | ((uint32_t)m1 << 16);
    *reinterpret_cast<uint32_t*>(D + (2 * ntp + t) * ld_pix + i0) =
        (uint32_t)a0 | ((uint32_t)a1 << 16);
  }
}

// bias_j = log w_j - (sum of the slices' partial sums, in slice order); with
// the last iteration's bias, the tile's largest rise and fall of it into
// bpm[t], bpm[nt + t] (rounded up). One CTA of 128 threads per row tile.
__global__ void __launch_bounds__(kTRows)
    expand_bias_kernel(const double* __restrict__ partial, int n_slices, int64_t rows,
                       const double* __restrict__ logw, int64_t nrot, double* __restrict__ bias,
                       const double* __restrict__ bias_old, float* __restrict__ bpm, int64_t nt) {
  __shared__ double rp[kTRows], rm[kTRows];
  const int64_t row = (int64_t)blockIdx.x * kTRows + threadIdx.x;
  double s = 0.0;
  for (int c = 0; c < n_slices; c++) s += partial[(int64_t)c * rows + row];
  const bool v = row < nrot;
  const double b = v ? logw[row] - s : -INFINITY;
  bias[row] = b;
  if (!bias_old) return;
  const double d = v ? b - bias_old[row] : 0.0;
  rp[threadIdx.x] = v ? d : -INFINITY;
  rm[threadIdx.x] = v ? -d : -INFINITY;
  __syncthreads();
  for (int w = kTRows / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      rp[threadIdx.x] = fmax(rp[threadIdx.x], rp[threadIdx.x + w]);
      rm[threadIdx.x] = fmax(rm[threadIdx.x], rm[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bpm[blockIdx.x] = __double2float_ru(rp[0]);
    bpm[nt + blockIdx.x] = __double2float_ru(rm[0]);
  }
}

// the grid in the corner-pair layout of trilinear_g4
__global__ void grid_pairs_kernel(const float* __restrict__ g, int N, float4* __restrict__ g4) {
  const int64_t n3 = (int64_t)N * N * N;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n3) return;
  const int z = (int)(l % N), y = (int)((l / N) % N);
  const bool zi = z + 1 < N, yi = y + 1 < N;
  g4[l] = make_float4(g[l], zi ? g[l + 1] : 0.f, yi ? g[l + N] : 0.f,
                      (zi && yi) ? g[l + N + 1] : 0.f);
}

// fixed-point pixel geometry from the double-float one
__global__ void fixed_geometry_kernel(const float4* __restrict__ qh, const float4* __restrict__ ql,
                                      int64_t ld_pix, int4* __restrict__ qi,
                                      float4* __restrict__ qlo, float4* __restrict__ qf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ld_pix) return;
  const float4 a = qh[i], b = ql[i];
  const double q[3] = {(double)a.x + (double)b.x, (double)a.y + (double)b.y,
                       (double)a.z + (double)b.z};
  int h[3];
  float l[3];
  for (int c = 0; c < 3; c++) {
    const double r = rint(q[c] * 4096.0);
    h[c] = (int)r;
    l[c] = (float)(q[c] - r / 4096.0);
  }
  qi[i] = make_int4(h[0], h[1], h[2], (int)a.w);
  qlo[i] = make_float4(l[0], l[1], l[2], 0.f);
  if (qf) qf[i] = make_float4((float)h[0] * 0x1p-12f, (float)h[1] * 0x1p-12f,
                              (float)h[2] * 0x1p-12f, 0.f);
}

}  // namespace

int64_t expand_tile_slices(int64_t ld_pix) { return (ld_pix + kTPix - 1) / kTPix; }

cudaError_t launch_grid_pairs(const float* grid, int N, float4* g4, cudaStream_t s) {
  const int64_t n3 = (int64_t)N * N * N;
  grid_pairs_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(grid, N, g4);
  return cudaGetLastError();
}

cudaError_t launch_fixed_geometry(const float4* qh, const float4* ql, int64_t ld_pix, int4* qi,
                                  float4* qlo, float4* qf, cudaStream_t s) {
  fixed_geometry_kernel<<<(unsigned)((ld_pix + 255) / 256), 256, 0, s>>>(qh, ql, ld_pix, qi, qlo,
                                                                        qf);
  return cudaGetLastError();
}

cudaError_t launch_expand_tile(const Geom& g, const float* grid, const float4* g4,
                               const RotFX* rot,
                               const double* logw, int64_t nrot, int64_t rows, int precision,
                               float w_floor, Planes L, double* bias, double* partial,
                               const void* Lold, const double* bias_old, uint16_t* D, int64_t ntp,
                               float* bpm, int32_t* status, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const int64_t nt = rows / kTRows;
  const int64_t ns = expand_tile_slices(g.ld_pix);
  const bool delta = Lold != nullptr;
  dim3 grd((unsigned)ns, (unsigned)nt);
#define EMC_TILE(P, I, DL)                                                                    \
  expand_tile_kernel<P, I, DL><<<grd, kTThreads, 0, s>>>(                                     \
      g.qi, g.qlo, g.ld_pix, g.N, grid, g4, rot, nrot, rows, w_floor, L.base, L.plane_stride, \
      partial, Lold, D, ntp, status)
#define EMC_TILE_P(P)                          \
  if (g.interior) {                            \
    if (delta) EMC_TILE(P, true, true);        \
    else EMC_TILE(P, true, false);             \
  } else {                                     \
    if (delta) EMC_TILE(P, false, true);       \
    else EMC_TILE(P, false, false);            \
  }
  switch (precision) {
    case EMC_PREC_FP32: EMC_TILE_P(EMC_PREC_FP32); break;
    case EMC_PREC_BF16: EMC_TILE_P(EMC_PREC_BF16); break;
    case EMC_PREC_FP16_SPLIT: EMC_TILE_P(EMC_PREC_FP16_SPLIT); break;
    default: EMC_TILE_P(EMC_PREC_BF16_SPLIT); break;
  }
#undef EMC_TILE_P
#undef EMC_TILE
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  expand_bias_kernel<<<(unsigned)nt, kTRows, 0, s>>>(partial, (int)ns, rows, logw, nrot, bias,
                                                     delta ? bias_old : nullptr, bpm, nt);
  return cudaGetLastError();
}

}  // namespace emc
