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
// Frames are kept in an order that groups them by the row tile of their best
// rotation (rotations are numbered along a space-filling curve, so a row tile
// is a compact region of SO(3)): the frames of a 256-frame tile then share
// their live row tiles. The order is that of the previous iteration's best
// tiles (a counting sort, stable, so deterministic); it only affects how
// many tiles are skipped, never the result.
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

// One CTA per 32 frames (lanes) x 8 strides of row tiles (warps): the threshold
// of each frame from the maxima over every row tile, then, for each row tile, a
// ballot over the warp's 32 frames; a tile with a frame above its threshold sets
// live[mt * nnt + nt] = 1 (live is zeroed first; eight CTAs share a frame tile).
__global__ void __launch_bounds__(256)
    bound_live_kernel(const double* __restrict__ part_m, int64_t n_mtiles, int64_t ld_data,
                      int64_t n_data, const float* __restrict__ nsum, float div,
                      uint8_t* __restrict__ live) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * 32 + lane;
  const int64_t nnt = ld_data / 256;
  const bool ok = s < n_data;
  double M = -INFINITY;
  if (ok)
    for (int64_t mt = r; mt < n_mtiles; mt += 8) M = fmax(M, part_m[mt * ld_data + s]);
  red[r][lane] = M;
  __syncthreads();
  double thr = INFINITY;  // padding frames never make a tile live
  if (ok) {
    M = red[0][lane];
    for (int q = 1; q < 8; q++) M = fmax(M, red[q][lane]);
    thr = M - (2.0 * ((double)nsum[s] / (double)div + 1.0) + 111.0);
  }
  for (int64_t mt = r; mt < n_mtiles; mt += 8) {
    const bool on = ok && part_m[mt * ld_data + s] >= thr;
    if (__any_sync(0xffffffffu, on) && lane == 0) live[mt * nnt + (s >> 8)] = 1;
  }
}

// One CTA: the live tiles in the raster order of the dense kernel (groups of
// `group` row tiles, frame tiles within a group, row tiles within those) into
// list, and their number into *count.
__global__ void __launch_bounds__(1024)
    tile_list_kernel(const uint8_t* __restrict__ live, int n_mtiles, int n_ntiles, int group,
                     int32_t* __restrict__ list, int32_t* __restrict__ count) {
  __shared__ int wsum[32];
  __shared__ int base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) base = 0;
  __syncthreads();
  const int T = n_mtiles * n_ntiles;
  const int per_group = group * n_ntiles;
  for (int t0 = 0; t0 < T; t0 += 1024) {
    const int t = t0 + tid;
    int code = 0;
    bool on = false;
    if (t < T) {
      const int g = t / per_group, rem = t % per_group;
      const int gsize = min(group, n_mtiles - g * group);
      const int nt = rem / gsize, mt = g * group + rem % gsize;
      code = mt * n_ntiles + nt;
      on = live[code] != 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 32; w++) {
      before += w < wid ? wsum[w] : 0;
      total += wsum[w];
    }
    if (on) list[base + before + __popc(m & ((1u << lane) - 1u))] = code;
    __syncthreads();
    if (tid == 0) base += total;
    __syncthreads();
  }
  if (tid == 0) *count = base;
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

cudaError_t launch_bound_live(const double* part_m, int64_t n_mtiles, int64_t ld_data,
                              int64_t n_data, const float* nsum, float div, uint8_t* live,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(live, 0, (size_t)n_mtiles * (ld_data / 256), s);
  if (e != cudaSuccess) return e;
  bound_live_kernel<<<(unsigned)(ld_data / 32), 256, 0, s>>>(part_m, n_mtiles, ld_data, n_data,
                                                              nsum, div, live);
  return cudaGetLastError();
}

cudaError_t launch_tile_list(const uint8_t* live, int n_mtiles, int n_ntiles, int group,
                             int32_t* list, int32_t* count, cudaStream_t s) {
  tile_list_kernel<<<1, 1024, 0, s>>>(live, n_mtiles, n_ntiles, group, list, count);
  return cudaGetLastError();
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

}  // namespace emc
