// prune.cu -- exact pruning of the E-step pass 1 inside emc_iteration.
//
// The BF16 three-term split writes log W = hi + mid + lo with hi on the 1/8
// grid and |mid + lo| <= 1/16 (plus 2^-16 of it); the FP16 split, hi on the
// 1/64 grid and |rest| <= 1/128. A contraction of the hi plane alone gives,
// for every (j, k), S^hi_jk = sum_i K_ik hi_ij + bias_j with
//   |S_jk - S^hi_jk| <= E_k = N_k / div + 1,   N_k = sum_i K_ik
// (div = 16 or 128; one unit covers the bias rest and every rounding). A row tile t whose
// maximum of S^hi over its rows, for frame k, lies below
//   M^hi_k - 2 E_k - 111,   M^hi_k = max_j S^hi_jk,
// has every S_jk < max_j S_jk - 110: its responsibilities e^(S - lse) are
// below e^-110 (< 2^-158), exactly 0 in FP32, and its share of the
// log-sum-exp sum is below FP64's rounding of the rest. Such (row tile,
// frame tile) pairs are skipped by the exact contraction; lse and P are those
// of the full one.
//
// In general terms: with an upper bound Ub_tk >= max_{j in t} S_jk for every
// row tile and a lower bound Lk <= max_j S_jk, a tile with Ub_tk < Lk - 111
// for every frame of a frame tile is skipped. Three stages give the bounds:
//  1. from the last iteration on the same frames (its exact tile maxima and
//     bounds, kept in Ub): the incremental bound below, for every tile, at
//     1/128 of the hi-plane contraction's work;
//  2. the hi-plane contraction over the pairs of row tiles that stage 1 could
//     not rule out (every pair on the first pruned pass, or after new frames):
//     Ub = min(Ub, S^hi max + E_k), Lk = max(Lk, S^hi max - E_k);
//  3. the exact three-plane contraction of the tiles left live, whose maxima
//     (plus 1/64) replace their bounds for the next iteration.
//
// Frames are kept in an order that groups them by the row tile of their best
// rotation (rotations are numbered along a space-filling curve, so a row tile
// is a compact region of SO(3)): the frames of a 256-frame tile then share
// their live row tiles. The order is that of the previous iteration's best
// tiles (a counting sort, stable, so deterministic); it only affects how
// many tiles are skipped, never the result.
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

// The live tiles in the raster order of the dense kernel (groups of `group`
// row tiles, frame tiles within a group, row tiles within those) into list,
// and their number into *count. Three launches: per CTA of kListChunk raster
// positions the number of live tiles; an exclusive scan of those numbers (in
// place, in the scratch `cnt`, one entry per CTA); per CTA the codes written
// from its offset on, each thread its kListItems consecutive positions after a
// block-wide scan of the threads' numbers. The order is the raster order.
constexpr int kListThreads = 1024;
constexpr int kListItems = 8;
constexpr int kListChunk = kListThreads * kListItems;

__device__ __forceinline__ int raster_code(int t, int n_mtiles, int n_ntiles, int group) {
  const int per_group = group * n_ntiles;
  const int g = t / per_group, rem = t % per_group;
  const int gsize = min(group, n_mtiles - g * group);
  const int nt = rem / gsize, mt = g * group + rem % gsize;
  return mt * n_ntiles + nt;
}

// live flags of the thread's positions as bits; their number
__device__ __forceinline__ unsigned list_bits(const uint8_t* __restrict__ live, int n_mtiles,
                                              int n_ntiles, int group, int T, int t0) {
  unsigned bits = 0;
#pragma unroll
  for (int q = 0; q < kListItems; q++) {
    const int t = t0 + q;
    if (t < T && live[raster_code(t, n_mtiles, n_ntiles, group)]) bits |= 1u << q;
  }
  return bits;
}

// sum over the CTA (every thread gets it); sh: 32 ints
__device__ __forceinline__ int block_sum(int v, int* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int tot = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
  tot = __reduce_add_sync(0xffffffffu, tot);
  __syncthreads();
  return tot;
}

// exclusive prefix over the CTA in thread order; sh: 32 ints
__device__ __forceinline__ int block_exclusive(int v, int* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int before = wid > 0 ? sh[wid - 1] : 0;
  __syncthreads();
  return before + inc - v;
}

__global__ void __launch_bounds__(kListThreads)
    tile_count_kernel(const uint8_t* __restrict__ live, int n_mtiles, int n_ntiles, int group,
                      int T, int32_t* __restrict__ cnt) {
  __shared__ int sh[32];
  const int t0 = blockIdx.x * kListChunk + threadIdx.x * kListItems;
  const int n = __popc(list_bits(live, n_mtiles, n_ntiles, group, T, t0));
  const int tot = block_sum(n, sh);
  if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

// one CTA: cnt[0 .. nb) to exclusive offsets, their total into *count
__global__ void __launch_bounds__(kListThreads)
    tile_scan_kernel(int32_t* __restrict__ cnt, int nb, int32_t* __restrict__ count) {
  __shared__ int sh[32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kListThreads) {
    const int b = b0 + threadIdx.x;
    const int v = b < nb ? cnt[b] : 0;
    const int ex = block_exclusive(v, sh);
    const int tot = block_sum(v, sh);
    if (b < nb) cnt[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(kListThreads)
    tile_write_kernel(const uint8_t* __restrict__ live, int n_mtiles, int n_ntiles, int group,
                      int T, const int32_t* __restrict__ off, int32_t* __restrict__ list) {
  __shared__ int sh[32];
  const int t0 = blockIdx.x * kListChunk + threadIdx.x * kListItems;
  unsigned bits = list_bits(live, n_mtiles, n_ntiles, group, T, t0);
  int pos = off[blockIdx.x] + block_exclusive(__popc(bits), sh);
  while (bits) {
    const int q = __ffs(bits) - 1;
    bits &= bits - 1;
    list[pos++] = raster_code(t0 + q, n_mtiles, n_ntiles, group);
  }
}

// Counting sort of the frames by key (their best row tile), stable: per chunk
// of 1024 frames a histogram H[bin * n_chunks + chunk] ...
__global__ void __launch_bounds__(1024)
    sort_hist_kernel(const int32_t* __restrict__ key, int64_t n_data, int nbins, int n_chunks,
                     int32_t* __restrict__ H) {
  extern __shared__ int hist[];
  const int chunk = blockIdx.x;
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const int64_t s = (int64_t)chunk * 1024 + threadIdx.x;
  if (s < n_data) atomicAdd(&hist[key[s]], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) H[(int64_t)b * n_chunks + chunk] = hist[b];
}

// ... then, after an exclusive scan of H in (bin, chunk) order, every frame's
// new position is its bin-and-chunk offset plus its rank among the earlier
// frames of its chunk with the same key. new_perm[pos] = perm[s].
__global__ void __launch_bounds__(1024)
    sort_scatter_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ perm,
                        int64_t n_data, int n_chunks, const int64_t* __restrict__ off,
                        int32_t* __restrict__ new_perm) {
  __shared__ int keys[1024];
  const int chunk = blockIdx.x;
  const int64_t s = (int64_t)chunk * 1024 + threadIdx.x;
  const int k = s < n_data ? key[s] : -1;
  keys[threadIdx.x] = k;
  __syncthreads();
  if (s >= n_data) return;
  int rank = 0;
  for (int t = 0; t < (int)threadIdx.x; t++) rank += keys[t] == k;
  const int64_t pos = off[(int64_t)k * n_chunks + chunk] + rank;
  new_perm[pos] = perm[s];
}

// Frames in the new order: rows of the BF16 frame matrix, the frame totals and
// (Poisson-fluence model) the score shift and 1 / N_k; iperm[original] = position.
__global__ void __launch_bounds__(256)
    permute_frames_kernel(const int32_t* __restrict__ perm, int64_t ld_data, int64_t ld_pix,
                          const uint16_t* __restrict__ Kb, uint16_t* __restrict__ Kp,
                          const float* __restrict__ nsum, float* __restrict__ nsum_p,
                          const double* __restrict__ cn, double* __restrict__ cn_p,
                          const float* __restrict__ invn, float* __restrict__ invn_p,
                          int32_t* __restrict__ iperm) {
  const int64_t pos = blockIdx.x;
  const int64_t k = perm[pos];
  const uint4* src = reinterpret_cast<const uint4*>(Kb + k * ld_pix);
  uint4* dst = reinterpret_cast<uint4*>(Kp + pos * ld_pix);
  for (int64_t i = threadIdx.x; i < ld_pix / 8; i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) {
    nsum_p[pos] = nsum[k];
    if (cn) cn_p[pos] = cn[k];
    if (invn) invn_p[pos] = invn[k];
    iperm[k] = (int32_t)pos;
  }
}

// Frame totals N_k (original order; 0 for padding frames).
__global__ void __launch_bounds__(256)
    frame_totals_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                        int64_t n_pix, float* __restrict__ nsum) {
  const int64_t k = blockIdx.x;
  __shared__ long long red[8];
  long long n = 0;
  if (k < n_data)
    for (int64_t i = threadIdx.x; i < n_pix; i += blockDim.x) n += K[k * ld_k + i];
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < 8; w++) t += red[w];
    nsum[k] = (float)t;
  }
}

__global__ void identity_kernel(int32_t* __restrict__ p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

// lse of the sorted frames back to the original order.
__global__ void unpermute_lse_kernel(const int32_t* __restrict__ perm, int64_t n_data,
                                     const double* __restrict__ m_s, const double* __restrict__ s_s,
                                     double* __restrict__ m, double* __restrict__ s) {
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n_data) return;
  const int64_t k = perm[pos];
  m[k] = m_s[pos];
  s[k] = s_s[pos];
}

cudaError_t launch_tile_list(const uint8_t* live, int n_mtiles, int n_ntiles, int group,
                             int32_t* list, int32_t* count, int32_t* scratch, cudaStream_t s) {
  const int T = n_mtiles * n_ntiles;
  const int nb = (T + kListChunk - 1) / kListChunk;
  tile_count_kernel<<<nb, kListThreads, 0, s>>>(live, n_mtiles, n_ntiles, group, T, scratch);
  tile_scan_kernel<<<1, kListThreads, 0, s>>>(scratch, nb, count);
  tile_write_kernel<<<nb, kListThreads, 0, s>>>(live, n_mtiles, n_ntiles, group, T, scratch, list);
  return cudaGetLastError();
}

int64_t tile_list_scratch_entries(int64_t n_mtiles, int64_t n_ntiles) {
  return (n_mtiles * n_ntiles + kListChunk - 1) / kListChunk;
}

int64_t sort_scratch_entries(int64_t n_data, int nbins) {
  return (int64_t)nbins * ((n_data + 1023) / 1024);
}

cudaError_t launch_sort_frames(const int32_t* key, const int32_t* perm, int64_t n_data, int nbins,
                               int32_t* H, int64_t* off, int32_t* new_perm, cudaStream_t s) {
  const int n_chunks = (int)((n_data + 1023) / 1024);
  const size_t sm = sizeof(int) * (size_t)nbins;
  cudaError_t e = cudaSuccess;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(sort_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
  }
  sort_hist_kernel<<<n_chunks, 1024, sm, s>>>(key, n_data, nbins, n_chunks, H);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan_counts(H, (int64_t)nbins * n_chunks, off, s);
  if (e != cudaSuccess) return e;
  sort_scatter_kernel<<<n_chunks, 1024, 0, s>>>(key, perm, n_data, n_chunks, off, new_perm);
  return cudaGetLastError();
}

cudaError_t launch_permute_frames(const int32_t* perm, int64_t ld_data, int64_t ld_pix,
                                  const uint16_t* Kb, uint16_t* Kp, const float* nsum,
                                  float* nsum_p, const double* cn, double* cn_p, const float* invn,
                                  float* invn_p, int32_t* iperm, cudaStream_t s) {
  permute_frames_kernel<<<(unsigned)ld_data, 256, 0, s>>>(perm, ld_data, ld_pix, Kb, Kp, nsum,
                                                          nsum_p, cn, cn_p, invn, invn_p, iperm);
  return cudaGetLastError();
}

cudaError_t launch_frame_totals(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                int64_t ld_data, float* nsum, cudaStream_t s) {
  frame_totals_kernel<<<(unsigned)ld_data, 256, 0, s>>>(K, ld_k, n_data, n_pix, nsum);
  return cudaGetLastError();
}

cudaError_t launch_identity(int32_t* p, int64_t n, cudaStream_t s) {
  identity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_unpermute_lse(const int32_t* perm, int64_t n_data, const double* m_s,
                                 const double* s_s, double* m, double* s, cudaStream_t st) {
  unpermute_lse_kernel<<<(unsigned)((n_data + 255) / 256), 256, 0, st>>>(perm, n_data, m_s, s_s,
                                                                        m, s);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Incremental bound between consecutive iterations (same frames).
//
// With the three-term split, the represented log W of iteration n is
// L^n_ij = hi + mid + lo, and the scores S^n_jk = sum_i K_ik L^n_ij + bias^n_j.
// From one iteration to the next, for every j of row tile t,
//   S^{n+1}_jk - S^n_jk <= sum_i K_ik D+_ti + b+_t,
//   S^n_jk - S^{n+1}_jk <= sum_i K_ik D-_ti + b-_t,
// with D+_ti = max_{j in t} (L^{n+1}_ij - L^n_ij), D-_ti = max_{j in t}
// (L^n_ij - L^{n+1}_ij) (counts are non-negative) and b+-_t the same maxima of
// the bias change. D+- are rounded up to BF16 and contracted against the
// frames on the tensor cores (one row per tile: 1/128 of the hi-plane bound's
// work). The FP32 accumulation of sum_i K_ik D_ti errs by at most
// (ld_pix + 8) 2^-23 N_k max_i |D_ti| (products of an integer count <= 256
// and a BF16 value are exact in FP32; every addition rounds by at most one
// unit of 2^-23 of a partial sum, and every partial sum is bounded by
// sum_i K_ik A_ti, A_ti = max(|D+_ti|, |D-_ti|)), which is added: A is
// contracted with the increments, as a third block of rows.
// ---------------------------------------------------------------------------

// One plane value of L: BF16 or FP16 bits.
template <bool F16>
__device__ __forceinline__ float plane_val(const uint16_t* p, int64_t o) {
  if (F16) return __half2float(*reinterpret_cast<const __half*>(p + o));
  return __uint_as_float(((uint32_t)p[o]) << 16);
}
// The next BF16 (FP16) value >= x, as bits: the operand type of the frames.
template <bool F16>
__device__ __forceinline__ uint16_t round_up_bits(float x) {
  if (F16) {
    __half h = __float2half_ru(x);
    return *reinterpret_cast<uint16_t*>(&h);
  }
  __nv_bfloat16 b = __float2bfloat16_ru(x);
  return *reinterpret_cast<uint16_t*>(&b);
}

// One CTA per (pixel slice of 256 columns, row tile): each thread a pixel,
// the tile's valid rows in turn. D = [3 ntp][ld_pix]: rows t (D+), ntp + t
// (D-) and 2 ntp + t (A = max(|D+|, |D-|)), all rounded up to the frames'
// operand type; bpm[t], bpm[nt + t] = b+_t, b-_t (rounded up), written by the
// CTAs of the first slice.
template <int NP, bool F16>
__global__ void __launch_bounds__(256)
    delta_planes_kernel(const uint16_t* __restrict__ L0, const uint16_t* __restrict__ L1,
                        int64_t plane, int64_t ld_pix, int64_t nrot, const double* __restrict__ b0,
                        const double* __restrict__ b1, int64_t ntp, uint16_t* __restrict__ D,
                        float* __restrict__ bpm, int64_t nt) {
  const int64_t t = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t r0 = t * 128;
  const int64_t r1 = min(r0 + 128, nrot);
  float dp = -INFINITY, dm = -INFINITY;
  if (i < ld_pix) {
    for (int64_t j = r0; j < r1; j++) {
      const int64_t o = j * ld_pix + i;
      // the difference of each plane is exact in FP32; their sum rounds at most twice
      float d = plane_val<F16>(L1, o) - plane_val<F16>(L0, o);
#pragma unroll
      for (int q = 1; q < NP; q++) d += plane_val<F16>(L1, o + q * plane) - plane_val<F16>(L0, o + q * plane);
      dp = fmaxf(dp, d);
      dm = fmaxf(dm, -d);
    }
    // those roundings: 2^-23 |d| covers them
    dp += 2.0f * 1.1920929e-7f * fabsf(dp);
    dm += 2.0f * 1.1920929e-7f * fabsf(dm);
    const uint16_t up = round_up_bits<F16>(dp), um = round_up_bits<F16>(dm);
    D[t * ld_pix + i] = up;
    D[(ntp + t) * ld_pix + i] = um;
    // A bounds the magnitude of both rounded values
    D[(2 * ntp + t) * ld_pix + i] = round_up_bits<F16>(fmaxf(fabsf(dp), fabsf(dm)) * 1.0078125f);
  }
  if (blockIdx.x == 0 && threadIdx.x < 128) {
    __shared__ double rb[2][128];
    const int64_t j = r0 + threadIdx.x;
    const double db = j < nrot ? b1[j] - b0[j] : 0.0;
    rb[0][threadIdx.x] = j < nrot ? db : -INFINITY;
    rb[1][threadIdx.x] = j < nrot ? -db : -INFINITY;
    __syncwarp();
    for (int w = 64; w > 0; w >>= 1) {
      asm volatile("bar.sync 3, 128;" ::: "memory");
      if ((int)threadIdx.x < w) {
        rb[0][threadIdx.x] = fmax(rb[0][threadIdx.x], rb[0][threadIdx.x + w]);
        rb[1][threadIdx.x] = fmax(rb[1][threadIdx.x], rb[1][threadIdx.x + w]);
      }
    }
    if (threadIdx.x == 0) {
      bpm[t] = __double2float_ru(rb[0][0]);
      bpm[nt + t] = __double2float_ru(rb[1][0]);
    }
  }
}

// Per frame (lanes) and row tile (warp strides), with C = [D+; D-; A] K^T of
// the frames in the current internal order (rows t, ntp + t, 2 ntp + t):
//   Ub[t][k] += C+[t][k] + b+_t + err_tk        (err = errc (1 + errc) CA[t][k])
//   Lk[k] = Mk[k] - 1/64 - (C-[t*][k] + b-_t* + err_t*k),   t* = best[k]
// Mk: the last iteration's largest exact tile maximum (its scores are within
// 1/128 of it), t* its row tile, so Lk <= max_j S_jk now. A tile that this
// does not rule out (Ub >= Lk - 111) is a candidate for the hi-plane bound
// (cand[t][nt] = 1) only where that bound could do better: where the
// widening the incremental bound has gathered since the tile's bound was last
// refreshed (Ua, the C+ terms summed over iterations), plus this iteration's
// C- term, exceeds the hi-plane bound's 2 E_k = 2 (N_k / div + 1). Otherwise
// it goes to the exact pass. Both refresh the bound and clear Ua.
// invalid (host flag; changed[0], set by emc_set_frames when the counts
// differ from the last ones; or changed[2], the device status the last pass
// left): Ub = +inf, Lk = -inf and every tile a candidate.
__global__ void __launch_bounds__(256)
    delta_live_kernel(const float* __restrict__ C, int64_t ntp, const float* __restrict__ bpm,
                      float* __restrict__ Ub,
                      float* __restrict__ Ua, double* __restrict__ Lk,
                      const double* __restrict__ Mk,
                      const int32_t* __restrict__ best, const float* __restrict__ nsum,
                      double errc, float div, int64_t n_mtiles, int64_t ld_data,
                      int64_t n_data, int valid_host, const int32_t* __restrict__ changed,
                      uint8_t* __restrict__ cand) {
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * 32 + lane;
  const int64_t nnt = ld_data / 256;
  const bool ok = k < n_data;
  const bool valid = valid_host && !(changed && (changed[0] || changed[2]));
  // FP32 with upward rounding for the upper bounds (FP64 is rare on this part);
  // the frame's lower bound in FP64 once, then rounded down for the comparisons
  double L = -INFINITY;
  float wl = 0.f, Lf = -INFINITY;
  const float ec = __double2float_ru(errc);
  const float E2 = ok ? 2.f * (nsum[k] / div + 1.f) : 0.f;
  if (ok && valid) {
    const int tb = best[k];
    const float e = __fmul_ru(ec, C[(2 * ntp + tb) * ld_data + k]);
    wl = __fadd_ru(__fadd_ru(__fadd_ru(C[(ntp + tb) * ld_data + k], bpm[n_mtiles + tb]), e),
                   1.0f / 64.0f);
    L = Mk[k] - (double)wl;
    Lf = __double2float_rd(L - 111.0);
  }
  if (ok && r == 0) Lk[k] = L;
#pragma unroll 4
  for (int64_t t = r; t < n_mtiles; t += 8) {
    bool on = ok;
    if (ok) {
      float* u = Ub + t * ld_data + k;
      float* ua = Ua + t * ld_data + k;
      if (valid) {
        const float e = __fmul_ru(ec, C[(2 * ntp + t) * ld_data + k]);
        const float wu = __fadd_ru(__fadd_ru(C[t * ld_data + k], bpm[t]), e);
        const float U = __fadd_ru(*u, wu);
        const float acc = *ua + fmaxf(wu, 0.f);
        *u = U;
        *ua = acc;
        on = U >= Lf && acc + wl > E2;
      } else {
        *u = INFINITY;
        *ua = 0.f;
      }
    }
    if (__any_sync(0xffffffffu, on) && lane == 0) cand[t * nnt + (k >> 8)] = 1;
  }
}

// pf[mp][nt] = cand[2 mp][nt] | cand[2 mp + 1][nt]: the row-tile pairs the
// hi-plane bound contracts.
__global__ void pair_flags_kernel(const uint8_t* __restrict__ cand, int64_t n_mtiles, int64_t nnt,
                                  uint8_t* __restrict__ pf) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npairs = (n_mtiles + 1) / 2;
  if (x >= npairs * nnt) return;
  const int64_t mp = x / nnt, nt = x % nnt;
  uint8_t v = cand[2 * mp * nnt + nt];
  if (2 * mp + 1 < n_mtiles) v |= cand[(2 * mp + 1) * nnt + nt];
  pf[x] = v;
}

// Combination of both bounds and the liveness of every tile. For the tiles
// whose pair the hi-plane bound contracted (pf), part_m holds max_j S^hi over
// the tile, with |S - S^hi| <= E_k = N_k / div + 1:
//   Ub = min(Ub, part_m + E_k),   Lk = max(Lk, part_m - E_k).
// Then live[t][nt] = 1 where Ub >= Lk - 111 for some frame of the frame tile
// (live zeroed first): every score of a tile that is not live lies more than
// 111 below its frame's best (P = 0 in FP32, no weight in lse at FP64).
__global__ void __launch_bounds__(256)
    final_live_kernel(const double* __restrict__ part_m, const uint8_t* __restrict__ pf,
                      float* __restrict__ Ub, float* __restrict__ Ua, double* __restrict__ Lk,
                      const float* __restrict__ nsum, float div, int64_t n_mtiles,
                      int64_t ld_data, int64_t n_data, uint8_t* __restrict__ live) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * 32 + lane;
  const int64_t nnt = ld_data / 256;
  const bool ok = k < n_data;
  const double E = ok ? (double)nsum[k] / (double)div + 1.0 : 0.0;
  double L = ok ? Lk[k] : INFINITY;
  if (ok)
#pragma unroll 4
    for (int64_t t = r; t < n_mtiles; t += 8) {
      if (!pf[(t >> 1) * nnt + (k >> 8)]) continue;
      const double m = part_m[t * ld_data + k];
      float* u = Ub + t * ld_data + k;
      const float h = __double2float_ru(m + E);
      if (h < *u) {  // the hi-plane bound is the tighter one: refreshed
        *u = h;
        Ua[t * ld_data + k] = 0.f;
      }
      L = fmax(L, m - E);
    }
  red[r][lane] = L;
  __syncthreads();
  if (ok) {
    L = red[0][lane];
    for (int q = 1; q < 8; q++) L = fmax(L, red[q][lane]);
    if (r == 0) Lk[k] = L;
  }
  const float Lf = ok ? __double2float_rd(L - 111.0) : INFINITY;  // rounded down: safe side
#pragma unroll 4
  for (int64_t t = r; t < n_mtiles; t += 8) {
    const bool on = ok && Ub[t * ld_data + k] >= Lf;
    if (__any_sync(0xffffffffu, on) && lane == 0) live[t * nnt + (k >> 8)] = 1;
  }
}

// Per-frame state of the last iteration in a new internal order:
// src[pos] = iperm_old[perm_new[pos]] (the frame's old position).
__global__ void order_src_kernel(const int32_t* __restrict__ perm_new,
                                 const int32_t* __restrict__ iperm_old, int64_t n_data,
                                 int32_t* __restrict__ src) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_data) src[p] = iperm_old[perm_new[p]];
}

// Ub2[t][pos] = Ub[t][src[pos]] for every row tile (grid.y), and the row
// y == 0 also moves Mk and best.
__global__ void gather_state_kernel(const int32_t* __restrict__ src, int64_t n_data,
                                    int64_t ld_data, const float* __restrict__ Ub,
                                    float* __restrict__ Ub2, const float* __restrict__ Ua,
                                    float* __restrict__ Ua2, const double* __restrict__ Mk,
                                    double* __restrict__ Mk2, const int32_t* __restrict__ best,
                                    int32_t* __restrict__ best2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_data) return;
  const int64_t t = blockIdx.y;
  const int64_t q = src[p];
  Ub2[t * ld_data + p] = Ub[t * ld_data + q];
  Ua2[t * ld_data + p] = Ua[t * ld_data + q];
  if (t == 0) {
    Mk2[p] = Mk[q];
    best2[p] = best[q];
  }
}

// *flag = 1 where a frame's counts differ from the BF16 copy Kb already held
// (columns < n_pix; a count above 256 differs by construction). One CTA per frame.
__global__ void __launch_bounds__(256)
    frames_differ_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                         int64_t n_pix, const uint16_t* __restrict__ Kb, int64_t ld_pix, int fp16,
                         int32_t* __restrict__ flag) {
  const int64_t k = blockIdx.x;
  if (k >= n_data) return;
  int d = 0;
  for (int64_t i = threadIdx.x; i < n_pix; i += blockDim.x) {
    const uint16_t b = Kb[k * ld_pix + i];
    const float v = fp16 ? __half2float(*reinterpret_cast<const __half*>(&b))
                         : __uint_as_float(((uint32_t)b) << 16);
    d |= (float)K[k * ld_k + i] != v;
  }
  if (__syncthreads_or(d) && threadIdx.x == 0) *flag = 1;
}

cudaError_t launch_delta_planes(const uint16_t* L0, const uint16_t* L1, int64_t plane,
                                int64_t ld_pix, int64_t nrot, const double* b0, const double* b1,
                                int64_t ntp, uint16_t* D, float* bpm, int f16, cudaStream_t s) {
  const int64_t nt = (nrot + 127) / 128;
  dim3 grd((unsigned)((ld_pix + 255) / 256), (unsigned)nt);
  if (f16)  // FP16 split: hi + rest
    delta_planes_kernel<2, true><<<grd, 256, 0, s>>>(L0, L1, plane, ld_pix, nrot, b0, b1, ntp, D,
                                                     bpm, nt);
  else      // BF16 split: hi + mid + lo
    delta_planes_kernel<3, false><<<grd, 256, 0, s>>>(L0, L1, plane, ld_pix, nrot, b0, b1, ntp, D,
                                                      bpm, nt);
  return cudaGetLastError();
}

cudaError_t launch_delta_live(const float* C, int64_t ntp, const float* bpm,
                              float* Ub, float* Ua, double* Lk, const double* Mk,
                              const int32_t* best,
                              const float* nsum, float div, int64_t ld_pix, int64_t n_mtiles,
                              int64_t ld_data, int64_t n_data, int valid,
                              const int32_t* changed, uint8_t* cand, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cand, 0, (size_t)n_mtiles * (ld_data / 256), s);
  if (e != cudaSuccess) return e;
  // accumulation error per unit of sum_i K |D|, and the FP32 error of that sum itself
  const double ec = (double)(ld_pix + 8) * 0x1p-23;
  const double errc = ec * (1.0 + ec);
  delta_live_kernel<<<(unsigned)(ld_data / 32), 256, 0, s>>>(C, ntp, bpm, Ub, Ua, Lk, Mk, best,
                                                             nsum, errc, div, n_mtiles, ld_data,
                                                             n_data, valid, changed, cand);
  return cudaGetLastError();
}

cudaError_t launch_pair_flags(const uint8_t* cand, int64_t n_mtiles, int64_t nnt, uint8_t* pf,
                              cudaStream_t s) {
  const int64_t n = (n_mtiles + 1) / 2 * nnt;
  pair_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cand, n_mtiles, nnt, pf);
  return cudaGetLastError();
}

cudaError_t launch_final_live(const double* part_m, const uint8_t* pf, float* Ub, float* Ua,
                              double* Lk,
                              const float* nsum, float div, int64_t n_mtiles, int64_t ld_data,
                              int64_t n_data, uint8_t* live, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(live, 0, (size_t)n_mtiles * (ld_data / 256), s);
  if (e != cudaSuccess) return e;
  final_live_kernel<<<(unsigned)(ld_data / 32), 256, 0, s>>>(part_m, pf, Ub, Ua, Lk, nsum, div,
                                                             n_mtiles, ld_data, n_data, live);
  return cudaGetLastError();
}

cudaError_t launch_reorder_state(const int32_t* perm_new, const int32_t* iperm_old, int64_t n_data,
                                 int64_t ld_data, int64_t n_mtiles, int32_t* src, const float* Ub,
                                 float* Ub2, const float* Ua, float* Ua2, const double* Mk,
                                 double* Mk2, const int32_t* best, int32_t* best2,
                                 cudaStream_t s) {
  const unsigned nb = (unsigned)((n_data + 255) / 256);
  order_src_kernel<<<nb, 256, 0, s>>>(perm_new, iperm_old, n_data, src);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gather_state_kernel<<<dim3(nb, (unsigned)n_mtiles), 256, 0, s>>>(src, n_data, ld_data, Ub, Ub2,
                                                                   Ua, Ua2, Mk, Mk2, best, best2);
  return cudaGetLastError();
}

cudaError_t launch_frames_differ(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                 const uint16_t* Kb, int64_t ld_pix, int fp16, int32_t* flag,
                                 cudaStream_t s) {
  frames_differ_kernel<<<(unsigned)n_data, 256, 0, s>>>(K, ld_k, n_data, n_pix, Kb, ld_pix, fp16,
                                                        flag);
  return cudaGetLastError();
}

}  // namespace emc
