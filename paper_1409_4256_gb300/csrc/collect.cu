// collect.cu -- the non-zero responsibilities of an iteration, and the
// training targets and missed mass of the learned schedule drawn from them.
//
// P_jk = exp(S_jk - lse_k) (Eq. 2.4) is exactly 0 in FP32 for all but a few
// rotations per frame, and the pass that forms it already lists the 128 x 64
// blocks of P holding a non-zero value. After each rotation chunk's
// normalisation, collect_kernel reads those blocks from the chunk's P planes
// (the operand layout of the M-step: BF16 hi + lo, or FP16 hi + lo of 2^14 P;
// with the Poisson-fluence model P_jk B_j / N_k) and appends every non-zero
// (frame, rotation, P) to a caller-owned list. This needs no stored scores, so
// it also runs where they do not fit and pass 2 recomputes them.
//
// From the list, per frame (one warp each, in frame order):
//   * the R rotations of largest P with weights P / (sum of those R), i.e. the
//     softmax of their scores; rotations with P = 0 in FP32 (scores more than
//     about 103 below lse_k) have weight 0 and rank after every non-zero one,
//     so a frame with fewer than R non-zero entries is filled with distinct
//     rotations of weight 0 (from its best rotation's 128-rotation tile on);
//   * the missed mass of the frame's candidate set C_k: sum of P_jk over the
//     listed j outside C_k, i.e. 1 - sum_{j in C_k} P_jk up to the rounding of
//     the P planes (2^-16 relative for the two-term forms).
#include <limits.h>

#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

namespace {

constexpr int kColThreads = 256;

// P_jk of one element of the planes (see the file comment)
__device__ __forceinline__ float decode_p(uint16_t h, uint16_t l, int precision) {
  if (precision == EMC_PREC_FP16_SPLIT) return (fp16_val(h) + fp16_val(l)) * (1.0f / kP16Scale);
  return bf16_val(h) + bf16_val(l);
}

// One CTA per row tile of the chunk: its listed 64-frame blocks, 128 rows x
// 64 frames each; thread t reads frame column t mod 64 of rows t / 64 + 4 i.
__global__ void __launch_bounds__(kColThreads)
    collect_kernel(const uint16_t* __restrict__ P, int64_t plane, int64_t ld_data, int precision,
                   const double* __restrict__ Bsum, const float* __restrict__ invn, int64_t row0,
                   int64_t nr, const int32_t* __restrict__ kbc, const int32_t* __restrict__ kbl,
                   int kb_ld, const int32_t* __restrict__ perm, int64_t n_data,
                   unsigned long long* count, int32_t* __restrict__ ek, int32_t* __restrict__ ej,
                   float* __restrict__ ep, int64_t cap) {
  const int64_t mt = blockIdx.x;
  const int nb = kbc[mt];
  const int tid = threadIdx.x, lane = tid & 31;
  const int col = tid & 63, r_first = tid >> 6;
  for (int b = 0; b < nb; b++) {
    const int64_t k = (int64_t)kbl[mt * kb_ld + b] * 64 + col;  // frame position
    const bool kok = k < n_data;
    const float inv = (kok && invn) ? invn[k] : 1.0f;
#pragma unroll 4
    for (int i = 0; i < 32; i++) {
      const int r = r_first + 4 * i;
      const int64_t j = mt * 128 + r;  // row of the chunk
      float p = 0.f;
      if (kok && j < nr) {
        const int64_t o = j * ld_data + k;
        p = decode_p(P[o], P[o + plane], precision);
        if (Bsum && p != 0.f) p = (float)((double)p / (Bsum[j] * (double)inv));
      }
      const bool on = p > 0.f;
      const unsigned m = __ballot_sync(0xffffffffu, on);
      if (m == 0u) continue;
      unsigned long long base = 0ull;
      if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (on) {
        const unsigned long long e = base + __popc(m & ((1u << lane) - 1u));
        if (e < (unsigned long long)cap) {
          ek[e] = perm ? perm[k] : (int32_t)k;
          ej[e] = (int32_t)(row0 + j);
          ep[e] = p;
        }
      }
    }
  }
}

// entries per frame; a list that overflowed sets EMC_ERR_UNSUPPORTED
__global__ void collect_hist_kernel(const unsigned long long* count, int64_t cap,
                                    const int32_t* __restrict__ ek, int32_t* __restrict__ cnt,
                                    int32_t* status) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && *count > (unsigned long long)cap)
    set_status(status, EMC_ERR_UNSUPPORTED);
  const int64_t n = (int64_t)min(*count, (unsigned long long)cap);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + ek[e], 1);
}

// exclusive scan of cnt[0..n) into off[0..n] (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024)
    collect_scan_kernel(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ off) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + 1023) / 1024, a = t * per, b = min(n, a + per);
  int32_t s = 0;
  for (int64_t i = a; i < b; i++) s += cnt[i];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const int32_t v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - s;
  for (int64_t i = a; i < b; i++) {
    off[i] = run;
    run += cnt[i];
  }
  if (t == 1023) off[n] = part[1023];
}

__global__ void collect_scatter_kernel(const unsigned long long* count, int64_t cap,
                                       const int32_t* __restrict__ ek,
                                       const int32_t* __restrict__ ej,
                                       const float* __restrict__ ep,
                                       const int32_t* __restrict__ off, int32_t* __restrict__ fill,
                                       int32_t* __restrict__ sj, float* __restrict__ sp) {
  const int64_t n = (int64_t)min(*count, (unsigned long long)cap);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = ek[e];
    const int32_t at = off[k] + atomicAdd(fill + k, 1);
    sj[at] = ej[e];
    sp[at] = ep[e];
  }
}

// (p, j) ranks before (q, i): larger P first, then the lower rotation
__device__ __forceinline__ bool before(float p, int32_t j, float q, int32_t i) {
  return p > q || (p == q && j < i);
}

// One warp per frame: top R by repeated selection over the frame's entries
// (few: the rotations whose P is non-zero in FP32), the weights, the fill and
// the missed mass of the candidate set.
__global__ void collect_targets_kernel(const int32_t* __restrict__ off,
                                       const int32_t* __restrict__ sj,
                                       const float* __restrict__ sp, int64_t n_data, int64_t n_rot,
                                       int R, int32_t* __restrict__ tidx, float* __restrict__ tprob,
                                       const int32_t* __restrict__ cand, int n_cand,
                                       float* __restrict__ missed) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= n_data) return;
  const int32_t a = off[k], n = off[k + 1] - a;
  const int32_t* J = sj + a;
  const float* Pk = sp + a;
  int32_t* ti = tidx + k * R;
  float* tp = tprob + k * R;
  // selection: the r-th pick is the best entry ranking after the (r-1)-th
  float lp = INFINITY;
  int32_t lj = -1;
  float wsum = 0.f;
  int got = 0;
  for (int r = 0; r < R && r < n; r++) {
    float bp = -1.f;
    int32_t bj = INT_MAX;
    for (int e = lane; e < n; e += 32) {
      const float p = Pk[e];
      const int32_t j = J[e];
      if (before(lp, lj, p, j) && before(p, j, bp, bj)) {
        bp = p;
        bj = j;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float op = __shfl_xor_sync(0xffffffffu, bp, o);
      const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (before(op, oj, bp, bj)) {
        bp = op;
        bj = oj;
      }
    }
    if (lane == 0) {
      ti[r] = bj;
      tp[r] = bp;
    }
    wsum += bp;
    lp = bp;
    lj = bj;
    got++;
  }
  __syncwarp();
  for (int r = lane; r < got; r += 32) tp[r] = wsum > 0.f ? tp[r] / wsum : 0.f;
  // fill: distinct rotations of weight 0 from the best rotation's tile on
  if (got < R) {
    const int64_t start = got > 0 ? ((int64_t)ti[0] / 128) * 128 : 0;
    int have = got;
    for (int64_t s = 0; have < R && s < n_rot; s += 32) {
      const int64_t j = (start + s + lane) % n_rot;
      bool taken = s + lane >= n_rot;
      for (int r = 0; r < got && !taken; r++) taken = ti[r] == (int32_t)j;
      const unsigned m = __ballot_sync(0xffffffffu, !taken);
      const int pos = have + __popc(m & ((1u << lane) - 1u));
      if (!taken && pos < R) {
        ti[pos] = (int32_t)j;
        tp[pos] = 0.f;
      }
      have += __popc(m);
    }
  }
  if (missed) {
    float out = 0.f;
    const int32_t* C = cand + k * (int64_t)n_cand;
    for (int e = 0; e < n; e++) {  // few entries; the warp scans the set
      const int32_t j = J[e];
      bool in = false;
      for (int c = lane; c < n_cand && !in; c += 32) in = C[c] == j;
      if (!__any_sync(0xffffffffu, in)) out += Pk[e];
    }
    if (lane == 0) missed[k] = out;
  }
}

}  // namespace

size_t collect_layout(int64_t cap, int64_t n_data, CollectBuf* b, char* base) {
  size_t o = 256;  // the count first
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t ek = take(sizeof(int32_t) * cap), ej = take(sizeof(int32_t) * cap),
               ep = take(sizeof(float) * cap), sj = take(sizeof(int32_t) * cap),
               sp = take(sizeof(float) * cap), cnt = take(sizeof(int32_t) * (n_data + 1)),
               off = take(sizeof(int32_t) * (n_data + 1)), fill = take(sizeof(int32_t) * n_data);
  if (b && base) {
    b->count = (unsigned long long*)base;
    b->ek = (int32_t*)(base + ek);
    b->ej = (int32_t*)(base + ej);
    b->ep = (float*)(base + ep);
    b->sj = (int32_t*)(base + sj);
    b->sp = (float*)(base + sp);
    b->cnt = (int32_t*)(base + cnt);
    b->off = (int32_t*)(base + off);
    b->fill = (int32_t*)(base + fill);
    b->cap = cap;
  }
  return o;
}

cudaError_t launch_collect(const void* P, int64_t plane, int64_t ld_data, int precision,
                           const double* Bsum, const float* invn, int64_t row0, int64_t nr,
                           int64_t n_mtiles, const int32_t* kbc, const int32_t* kbl, int kb_ld,
                           const int32_t* perm, int64_t n_data, const CollectBuf& b,
                           cudaStream_t s) {
  if (n_mtiles <= 0) return cudaSuccess;
  collect_kernel<<<(unsigned)n_mtiles, kColThreads, 0, s>>>(
      (const uint16_t*)P, plane, ld_data, precision, Bsum, invn, row0, nr, kbc, kbl, kb_ld, perm,
      n_data, b.count, b.ek, b.ej, b.ep, b.cap);
  return cudaGetLastError();
}

cudaError_t launch_collected_targets(const CollectBuf& b, int64_t n_data, int64_t n_rot, int R,
                                     int32_t* tidx, float* tprob, const int32_t* cand, int n_cand,
                                     float* missed, int32_t* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * (n_data + 1), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(b.fill, 0, sizeof(int32_t) * n_data, s);
  if (e != cudaSuccess) return e;
  const unsigned g = 152 * 8;
  collect_hist_kernel<<<g, 256, 0, s>>>(b.count, b.cap, b.ek, b.cnt, status);
  collect_scan_kernel<<<1, 1024, 0, s>>>(b.cnt, n_data, b.off);
  collect_scatter_kernel<<<g, 256, 0, s>>>(b.count, b.cap, b.ek, b.ej, b.ep, b.off, b.fill, b.sj,
                                           b.sp);
  const int64_t threads = n_data * 32;
  collect_targets_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      b.off, b.sj, b.sp, n_data, n_rot, R, tidx, tprob, cand, n_cand, missed);
  return cudaGetLastError();
}

}  // namespace emc
