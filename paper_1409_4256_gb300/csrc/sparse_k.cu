// sparse_k.cu -- sparse-K form of the E-step pass 1 (the paper has no
// counterpart: an alternative contraction for frames with few photons).
//
// S_jk = sum_i K_ik log W_ij + bias_j (Eqs. 2.3-2.4, Poisson) only needs the
// pixels where K_ik > 0. The frames are kept as a list of non-zero pixels per
// frame (CSR: offsets int64[ld_data + 1], entries uint32 = pixel | count << 16,
// in pixel order), and log W is gathered at those pixels instead of being
// contracted densely on the tensor cores.
//
// Kernel: one CTA per 128-rotation tile x 256 frames. The rotation tile is
// staged R rows at a time in shared memory as (hi on the 1/8 grid, rest),
// the split of the FP32 SIMT form, so that the count x hi sums are exact in
// FP32; each warp owns 32 frames, its lanes stride over a frame's entries and
// gather from the staged rows, a warp reduction gives the R scores of the
// frame, and the frame's owner lane keeps a running (max, sum) over the
// tile's rotations with the max on the 1/64 grid (exact differences). The
// per-tile pairs are merged by lse_merge exactly as those of the dense pass.
//
// Cost per (rotation, frame) pair: one gather per non-zero pixel from shared
// memory, against 2 n_pix (x 3 split terms) FLOP on the tensor cores for the
// dense pass -- it only pays off for frames with a few percent non-zero pixels.
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

constexpr int kSkThreads = 256;
constexpr int kSkFrames = 256;  // frames per CTA (8 warps x 32)
constexpr int kSkRows = 128;    // rotations per CTA (one pass-1 tile)
constexpr float kSkSentinel = -3.0e38f;

// non-zero pixels per frame (0 for padding frames)
__global__ void frames_nnz_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                                  int64_t n_pix, int32_t* __restrict__ cnt) {
  const int64_t k = blockIdx.x;
  int c = 0;
  if (k < n_data)
    for (int64_t i = threadIdx.x; i < n_pix; i += blockDim.x) c += K[k * ld_k + i] > 0;
  c = __reduce_add_sync(0xffffffffu, (unsigned)c);
  __shared__ int red[kSkThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kSkThreads / 32; w++) s += red[w];
    cnt[k] = s;
  }
}

// ordered compaction of one frame's non-zero pixels (block-wide ballot scan)
__global__ void frames_fill_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                                   int64_t n_pix, const int64_t* __restrict__ off,
                                   uint32_t* __restrict__ ent) {
  const int64_t k = blockIdx.x;
  if (k >= n_data) return;
  __shared__ int wsum[kSkThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t base_out = off[k];
  for (int64_t base = 0; base < n_pix; base += kSkThreads) {
    const int64_t i = base + threadIdx.x;
    const int32_t c = i < n_pix ? K[k * ld_k + i] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, c > 0);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kSkThreads / 32; w++) {
      before += w < warp ? wsum[w] : 0;
      total += wsum[w];
    }
    if (c > 0)
      ent[base_out + before + __popc(m & ((1u << lane) - 1u))] =
          (uint32_t)i | ((uint32_t)c << 16);
    base_out += total;
    __syncthreads();
  }
}

// One CTA per (256-frame block, 128-rotation tile); R rows staged at a time.
__global__ void __launch_bounds__(kSkThreads)
    sparse_k_pass1_kernel(const float* __restrict__ L, int64_t ld_pix, int64_t n_pix,
                          const double* __restrict__ bias, const int64_t* __restrict__ off,
                          const uint32_t* __restrict__ ent, int64_t ld_data, int64_t n_data,
                          int R, double* __restrict__ part_m, float* __restrict__ part_s) {
  extern __shared__ float sk_smem[];
  float* Lh = sk_smem;               // [R][ld_pix]
  float* Lr = sk_smem + R * ld_pix;  // [R][ld_pix]
  __shared__ float sbh[8], sbl[8];
  __shared__ int sval[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j_tile = (int64_t)blockIdx.y * kSkRows;
  const int64_t k_own = (int64_t)blockIdx.x * kSkFrames + warp * 32 + lane;  // lane's frame
  float run_m = kSkSentinel, run_s = 0.f;  // running (max on the 1/64 grid, sum) of k_own
  for (int g = 0; g < kSkRows; g += R) {
    __syncthreads();  // the previous group's rows are no longer read
    for (int r = 0; r < R; r++) {
      const int64_t j = j_tile + g + r;
      for (int64_t i = threadIdx.x; i < n_pix; i += kSkThreads) {
        const float x = L[j * ld_pix + i];
        const float h = rintf(x * kHiScale) * (1.0f / kHiScale);
        Lh[r * ld_pix + i] = h;
        Lr[r * ld_pix + i] = x - h;
      }
      if (threadIdx.x == 0) {
        const double b = bias[j];
        const bool v = b > -INFINITY;
        const float bh = v ? (float)(rint(b * kGridD) / kGridD) : 0.f;
        sbh[r] = bh;
        sbl[r] = v ? (float)(b - (double)bh) : 0.f;
        sval[r] = v;
      }
    }
    __syncthreads();
    for (int f = 0; f < 32; f++) {
      const int64_t k = (int64_t)blockIdx.x * kSkFrames + warp * 32 + f;
      if (k >= n_data) break;  // uniform across the warp
      float ah[8], ar[8];
#pragma unroll
      for (int r = 0; r < 8; r++) ah[r] = ar[r] = 0.f;
      const int64_t e1 = off[k + 1];
      for (int64_t e = off[k] + lane; e < e1; e += 32) {
        const uint32_t w = ent[e];
        const int idx = (int)(w & 0xffffu);
        const float c = (float)(w >> 16);
#pragma unroll
        for (int r = 0; r < 8; r++) {
          if (r < R) {
            ah[r] = fmaf(c, Lh[r * ld_pix + idx], ah[r]);
            ar[r] = fmaf(c, Lr[r * ld_pix + idx], ar[r]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 8; r++) {
        if (r < R) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            ah[r] += __shfl_xor_sync(0xffffffffu, ah[r], o);
            ar[r] += __shfl_xor_sync(0xffffffffu, ar[r], o);
          }
        }
      }
      if (lane == f) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
          if (r < R && sval[r]) {
            float h = ah[r] + sbh[r];  // exact: both on the 1/64 grid
            float l = ar[r] + sbl[r];
            const float rr = rintf(l * kGrid) * (1.0f / kGrid);
            h += rr;
            l -= rr;
            if (h > run_m) {
              run_s = run_s * __expf(run_m - h) + __expf(l);
              run_m = h;
            } else {
              run_s += __expf((h - run_m) + l);
            }
          }
        }
      }
    }
  }
  if (k_own < ld_data) {
    const int64_t o = (int64_t)blockIdx.y * ld_data + k_own;
    part_m[o] = run_s > 0.f ? (double)run_m : -INFINITY;
    part_s[o] = run_s;
  }
}

cudaError_t launch_sparse_k_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                   int64_t ld_data, int32_t* cnt, int64_t* off, uint32_t* ent,
                                   cudaStream_t s) {
  frames_nnz_kernel<<<(unsigned)ld_data, kSkThreads, 0, s>>>(K, ld_k, n_data, n_pix, cnt);
  cudaError_t e = launch_scan_counts(cnt, ld_data, off, s);
  if (e != cudaSuccess) return e;
  frames_fill_kernel<<<(unsigned)ld_data, kSkThreads, 0, s>>>(K, ld_k, n_data, n_pix, off, ent);
  return cudaGetLastError();
}

int sparse_k_rows_per_stage(int64_t ld_pix) {
  // R rows of (hi, rest) in at most ~200 KB of shared memory; R divides 128
  int R = 8;
  while (R > 1 && (size_t)R * 2 * ld_pix * sizeof(float) > 200u * 1024u) R >>= 1;
  return R;
}

size_t sparse_k_smem(int64_t ld_pix) {
  return (size_t)sparse_k_rows_per_stage(ld_pix) * 2 * ld_pix * sizeof(float);
}

cudaError_t launch_sparse_k_pass1(const float* L, int64_t ld_pix, int64_t n_pix, const double* bias,
                                  int64_t rows, const int64_t* off, const uint32_t* ent,
                                  int64_t ld_data, int64_t n_data, double* part_m, float* part_s,
                                  cudaStream_t s) {
  const int R = sparse_k_rows_per_stage(ld_pix);
  const size_t smem = sparse_k_smem(ld_pix);
  if (smem > 220u * 1024u) return cudaErrorInvalidValue;  // one row does not fit
  cudaError_t e = cudaFuncSetAttribute(sparse_k_pass1_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(ld_data / kSkFrames), (unsigned)(rows / kSkRows));
  sparse_k_pass1_kernel<<<grid, kSkThreads, smem, s>>>(L, ld_pix, n_pix, bias, off, ent, ld_data,
                                                      n_data, R, part_m, part_s);
  return cudaGetLastError();
}

}  // namespace emc
