// sparse.cu -- candidate selection and the Maximize step over candidate sets.
//
// Given M candidate rotations C_k per frame (from the learned proposal), the
// E- and M-steps (Eq. 2.4, 2.11) run over the pairs (j, k), j in C_k, only:
//   S_jk = sum_i K_ik log W_ij + bias_j,  lse_k = log sum_{j in C_k} exp S_jk,
//   P_jk = exp(S_jk - lse_k),  Num_j = sum_{k: j in C_k} P_jk K_k.
// The pairs are transposed once into a CSR list per rotation, so that both
// contractions read one log W row (staged in shared memory) and gather the
// frames' rows of K, which are 3x smaller than a split log W row and stay in L2
// at the 64^3 size. Scores use the same exact split as the dense forms (hi on
// the 1/8 grid accumulated exactly, a small residual).
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

// ------------------------------------------------------------------- top-M --
__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Block-wide exclusive prefix of a 0/1 flag (blockDim.x == 256); returns the
// prefix and writes the block total to *total.
__device__ __forceinline__ int block_prefix(int flag, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  const int in_warp = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) warp_tot[wid] = __popc(bal);
  __syncthreads();
  int before = 0, tot = 0;
  for (int w = 0; w < 8; w++) {
    if (w < wid) before += warp_tot[w];
    tot += warp_tot[w];
  }
  __syncthreads();
  *total = tot;
  return before + in_warp;
}

// One CTA (256 threads) per row: radix selection of the M-th largest key over
// four 8-bit digits, then the keys above it in index order followed by the
// first equal keys in index order (ties towards the lower index).
__global__ void __launch_bounds__(256)
    topm_kernel(const float* __restrict__ logits, int64_t ld, int n, int M,
                int32_t* __restrict__ cand) {
  const float* z = logits + (int64_t)blockIdx.x * ld;
  int32_t* out = cand + (int64_t)blockIdx.x * M;
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_mask;
  __shared__ int s_need;
  __shared__ int warp_tot[8];
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_mask = 0;
    s_need = M;
  }
  for (int shift = 24; shift >= 0; shift -= 8) {
    hist[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t prefix = s_prefix, mask = s_mask;
    for (int j = threadIdx.x; j < n; j += 256) {
      const uint32_t k = order_key(z[j]);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int cum = 0;
      for (int b = 255; b >= 0; b--) {
        if (cum + (int)hist[b] >= s_need) {
          s_prefix = prefix | ((uint32_t)b << shift);
          s_need -= cum;
          break;
        }
        cum += (int)hist[b];
      }
      s_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  const uint32_t T = s_prefix;
  const int need = s_need;  // how many keys equal to T are taken
  int gt_before = 0, eq_before = 0;
  for (int base = 0; base < n; base += 256) {
    const int j = base + threadIdx.x;
    const uint32_t k = j < n ? order_key(z[j]) : 0u;
    const int gt = j < n && k > T, eq = j < n && k == T;
    int tgt, teq;
    const int pg = block_prefix(gt, warp_tot, &tgt);
    const int pe = block_prefix(eq, warp_tot, &teq);
    if (gt) out[gt_before + pg] = j;
    if (eq && eq_before + pe < need) out[(M - need) + eq_before + pe] = j;
    gt_before += tgt;
    eq_before += teq;
  }
}

cudaError_t launch_topm(const float* logits, int64_t B, int64_t n, int64_t ld, int M,
                        int32_t* cand, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  topm_kernel<<<(unsigned)B, 256, 0, s>>>(logits, ld, (int)n, M, cand);
  return cudaGetLastError();
}

// ------------------------------------------------- training targets (top R) --
// Per frame (one thread, reading its frame-major scores sequentially): the R
// largest stored dense scores over rows [0, nrot) and their softmax
// (targets proportional to the dense responsibilities). iperm (may be NULL):
// the scores are in emc_iteration's internal frame order, frame k in column
// iperm[k]; live (may be NULL): only the row tiles t with
// live[t * (ld / 256) + column / 256] were contracted (the others hold no score).
__global__ void topr_columns_kernel(const float* __restrict__ S, int64_t ldS,
                                    const float* __restrict__ Sref, int64_t ld, int64_t nrot,
                                    int64_t n_data, int R, const int32_t* __restrict__ iperm,
                                    const uint8_t* __restrict__ live,
                                    int32_t* __restrict__ tidx, float* __restrict__ tprob) {
  const int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= n_data) return;
  const int64_t k = iperm ? iperm[kk] : kk;  // the score column
  const uint8_t* lv = live ? live + (k >> 8) : nullptr;
  const int64_t nnt = ld >> 8;
  float val[kMaxTargets];
  int idx[kMaxTargets];
  for (int r = 0; r < R; r++) {
    val[r] = -INFINITY;
    idx[r] = 0;
  }
  int mpos = 0;
  float mval = -INFINITY;
  for (int64_t j = 0; j < nrot; j++) {
    if (lv && !lv[(j >> 7) * nnt]) {
      j |= 127;  // a tile not contracted: its scores underflow next to the frame's best
      continue;
    }
    const float v = S[k * ldS + j] + Sref[(j >> 5) * ld + k];
    if (v > mval) {
      val[mpos] = v;
      idx[mpos] = (int)j;
      mval = val[0];
      mpos = 0;
      for (int r = 1; r < R; r++)
        if (val[r] < mval) {
          mval = val[r];
          mpos = r;
        }
    }
  }
  float mx = -INFINITY;
  for (int r = 0; r < R; r++) mx = fmaxf(mx, val[r]);
  float sum = 0.f;
  for (int r = 0; r < R; r++) sum += __expf(val[r] - mx);
  for (int r = 0; r < R; r++) {
    tidx[kk * R + r] = idx[r];
    tprob[kk * R + r] = __expf(val[r] - mx) / sum;
  }
}

cudaError_t launch_topr_columns(const float* S, int64_t ldS, const float* Sref, int64_t ld,
                                int64_t nrot, int64_t n_data, int R, int32_t* tidx, float* tprob,
                                cudaStream_t s, const int32_t* iperm, const uint8_t* live) {
  if (R < 1 || R > kMaxTargets) return cudaErrorInvalidValue;
  topr_columns_kernel<<<(unsigned)((n_data + 127) / 128), 128, 0, s>>>(
      S, ldS, Sref, ld, nrot, n_data, R, iperm, live, tidx, tprob);
  return cudaGetLastError();
}

// --------------------------------------------------------- CSR by rotation --
__global__ void csr_count_kernel(const int32_t* __restrict__ cand, int64_t n_pairs,
                                 int64_t n_rot, int32_t* __restrict__ cnt, int32_t* status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_pairs) return;
  const int32_t j = cand[e];
  if (j < 0 || j >= n_rot) {
    set_status(status, EMC_ERR_ARG);
    return;
  }
  atomicAdd(&cnt[j], 1);
}

// exclusive scan of cnt[0, n) into off[0, n] with one CTA of 1024 threads
__global__ void csr_scan_kernel(const int32_t* __restrict__ cnt, int64_t n,
                                int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  const int64_t per = (n + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = min(n, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; i++) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int t = 0; t < 1024; t++) {
      const int64_t v = part[t];
      part[t] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[threadIdx.x];
  for (int64_t i = b; i < e; i++) {
    off[i] = acc;
    acc += cnt[i];
  }
}

__global__ void csr_fill_kernel(const int32_t* __restrict__ cand, int64_t n_pairs, int M,
                                const int64_t* __restrict__ off, int32_t* __restrict__ cur,
                                int2* __restrict__ ent) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_pairs) return;
  const int32_t j = cand[e];
  const int64_t pos = off[j] + atomicAdd(&cur[j], 1);
  ent[pos] = make_int2((int)(e / M), (int)(e % M));
}

// Candidate sets from two ranked lists per frame: the R entries of `first`
// (distinct; the dense E-step's top R), then the entries of `rest` (the
// network's top list) that are not among them, in order, until M are written.
// With M_rest >= M at most R entries of rest repeat first, so M are always
// found. One warp per frame; membership by broadcasting first's entries.
__global__ void merge_candidates_kernel(const int32_t* __restrict__ first, int R,
                                        const int32_t* __restrict__ rest, int M_rest,
                                        int64_t n, int M, int32_t* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const int32_t* f = first + k * R;
  const int32_t* r = rest + k * M_rest;
  int32_t* o = out + k * M;
  const int32_t f0 = lane < R ? f[lane] : -1;
  const int32_t f1 = lane + 32 < R ? f[lane + 32] : -1;
  const int nf = R < M ? R : M;
  for (int t = lane; t < nf; t += 32) o[t] = f[t];
  int filled = nf;
  for (int base = 0; base < M_rest && filled < M; base += 32) {
    const int32_t c = base + lane < M_rest ? r[base + lane] : -1;
    bool dup = c < 0;
    for (int t = 0; t < R; t++) {
      const int32_t v = __shfl_sync(0xffffffffu, t < 32 ? f0 : f1, t & 31);
      dup |= v == c;
    }
    const unsigned keep = __ballot_sync(0xffffffffu, !dup);
    const int pos = filled + __popc(keep & ((1u << lane) - 1u));
    if (!dup && pos < M) o[pos] = c;
    filled += __popc(keep);
  }
}

cudaError_t launch_merge_candidates(const int32_t* first, int R, const int32_t* rest, int M_rest,
                                    int64_t n, int M, int32_t* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  merge_candidates_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(first, R, rest, M_rest, n, M,
                                                                  out);
  return cudaGetLastError();
}

cudaError_t launch_scan_counts(const int32_t* cnt, int64_t n, int64_t* off, cudaStream_t s) {
  csr_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, off);
  return cudaGetLastError();
}

cudaError_t launch_csr_build(const int32_t* cand, int64_t n_data, int M, int64_t n_rot,
                             int64_t rows, int32_t* cnt, int64_t* off, int2* ent,
                             int32_t* status, cudaStream_t s) {
  const int64_t n_pairs = n_data * M;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * rows, s);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((n_pairs + 255) / 256);
  csr_count_kernel<<<blocks, 256, 0, s>>>(cand, n_pairs, n_rot, cnt, status);
  csr_scan_kernel<<<1, 1024, 0, s>>>(cnt, rows, off);
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * rows, s)) != cudaSuccess) return e;
  csr_fill_kernel<<<blocks, 256, 0, s>>>(cand, n_pairs, M, off, cnt, ent);
  return cudaGetLastError();
}

// ------------------------------------------------------ sparse contractions --
// two frame counts packed in 32 bits (BF16 or FP16 frames)
template <bool KF16>
__device__ __forceinline__ void unpack2(uint32_t w, float& lo, float& hi) {
  if (KF16) {
    lo = fp16_val((uint16_t)(w & 0xffffu));
    hi = fp16_val((uint16_t)(w >> 16));
  } else {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xffff0000u);
  }
}

// One CTA per rotation row: log W_j split into (hi on the 1/8 grid, rest) in
// shared memory; each warp takes pairs (frame, slot) of the row's list, two
// at a time, reading the frames' K rows 8 pixels (16 bytes) per lane.
// CSR: the frames' non-zero pixel lists (pixel | count << 16, EMC_FLAG_SPARSE_K)
// are read instead of their rows -- 4 bytes per non-zero pixel rather than 2
// bytes per pixel -- and gathered against the staged row; the count x hi sums
// stay exact (integral counts, hi on the 1/8 grid, frame totals below 2^16).
template <int PREC, bool CSR>
__global__ void __launch_bounds__(256)
    sparse_scores_kernel(const void* __restrict__ L, int64_t plane_stride, int64_t ld_pix,
                         const double* __restrict__ bias, const uint16_t* __restrict__ Kb,
                         const int64_t* __restrict__ off, const int2* __restrict__ ent, int M,
                         const int64_t* __restrict__ koff, const uint32_t* __restrict__ kent,
                         double* __restrict__ Sc) {
  const int64_t j = blockIdx.x;
  const int64_t e0 = off[j], e1 = off[j + 1];
  if (e0 == e1) return;
  extern __shared__ float4 sm4[];
  float* Lh = reinterpret_cast<float*>(sm4);
  float* Lr = Lh + ld_pix;
  for (int64_t i = threadIdx.x; i < ld_pix; i += blockDim.x) {
    float h, r;
    if (PREC == EMC_PREC_FP32) {
      const float x = reinterpret_cast<const float*>(L)[j * ld_pix + i];
      h = rintf(x * 8.f) * 0.125f;
      r = x - h;
    } else if (PREC == EMC_PREC_FP16_SPLIT) {
      const uint16_t* Lb = reinterpret_cast<const uint16_t*>(L) + j * ld_pix + i;
      h = fp16_val(Lb[0]);
      r = fp16_val(Lb[plane_stride]);
    } else {
      const uint16_t* Lb = reinterpret_cast<const uint16_t*>(L) + j * ld_pix + i;
      h = bf16_val(Lb[0]);
      r = PREC == EMC_PREC_BF16_SPLIT ? bf16_val(Lb[plane_stride]) + bf16_val(Lb[2 * plane_stride])
                                      : 0.f;
    }
    Lh[i] = h;
    Lr[i] = r;
  }
  __syncthreads();
  const double bj = bias[j];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (CSR) {
    for (int64_t e = e0 + wid; e < e1; e += nw) {
      const int2 km = ent[e];
      const int64_t f1 = koff[km.x + 1];
      float ah = 0.f, ar = 0.f;
      for (int64_t f = koff[km.x] + lane; f < f1; f += 32) {
        const uint32_t w = kent[f];
        const int idx = (int)(w & 0xffffu);
        const float c = (float)(w >> 16);
        ah = fmaf(c, Lh[idx], ah);
        ar = fmaf(c, Lr[idx], ar);
      }
      for (int o = 16; o; o >>= 1) {
        ah += __shfl_xor_sync(0xffffffffu, ah, o);
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
      }
      if (lane == 0) Sc[(int64_t)km.x * M + km.y] = ((double)ah + (double)ar) + bj;
    }
    return;
  }
  const int64_t n8 = ld_pix / 8;
  for (int64_t e = e0 + 2 * wid; e < e1; e += 2 * nw) {
    const bool two = e + 1 < e1;
    const int2 ka = ent[e];
    const int2 kb = two ? ent[e + 1] : ka;
    const uint4* Ka = reinterpret_cast<const uint4*>(Kb + (int64_t)ka.x * ld_pix);
    const uint4* Kc = reinterpret_cast<const uint4*>(Kb + (int64_t)kb.x * ld_pix);
    float ah = 0.f, ar = 0.f, bh = 0.f, br = 0.f;
    for (int64_t g = lane; g < n8; g += 32) {
      const uint4 wa = Ka[g], wb = Kc[g];
      const float4 h0 = reinterpret_cast<const float4*>(Lh)[2 * g];
      const float4 h1 = reinterpret_cast<const float4*>(Lh)[2 * g + 1];
      const float4 r0 = reinterpret_cast<const float4*>(Lr)[2 * g];
      const float4 r1 = reinterpret_cast<const float4*>(Lr)[2 * g + 1];
      const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
      const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
      const uint32_t ua[4] = {wa.x, wa.y, wa.z, wa.w}, ub[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
      for (int c = 0; c < 4; c++) {
        float a0, a1, b0, b1;
        unpack2<PREC == EMC_PREC_FP16_SPLIT>(ua[c], a0, a1);
        unpack2<PREC == EMC_PREC_FP16_SPLIT>(ub[c], b0, b1);
        ah = fmaf(a0, hv[2 * c], ah);
        ah = fmaf(a1, hv[2 * c + 1], ah);
        ar = fmaf(a0, rv[2 * c], ar);
        ar = fmaf(a1, rv[2 * c + 1], ar);
        bh = fmaf(b0, hv[2 * c], bh);
        bh = fmaf(b1, hv[2 * c + 1], bh);
        br = fmaf(b0, rv[2 * c], br);
        br = fmaf(b1, rv[2 * c + 1], br);
      }
    }
    for (int o = 16; o; o >>= 1) {
      ah += __shfl_xor_sync(0xffffffffu, ah, o);
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      bh += __shfl_xor_sync(0xffffffffu, bh, o);
      br += __shfl_xor_sync(0xffffffffu, br, o);
    }
    if (lane == 0) {
      Sc[(int64_t)ka.x * M + ka.y] = ((double)ah + (double)ar) + bj;
      if (two) Sc[(int64_t)kb.x * M + kb.y] = ((double)bh + (double)br) + bj;
    }
  }
}

// One warp per frame: lse over the frame's M candidates, P = exp(S - lse).
// shift (may be NULL): per-frame constant the scores carry (Poisson-fluence
// model), removed from the lse written out.
__global__ void sparse_lse_kernel(const double* __restrict__ Sc, int64_t n_data, int64_t ld_data,
                                  int M, float* __restrict__ Pc, double* __restrict__ lse_c,
                                  const double* __restrict__ shift, int32_t* status) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= ld_data) return;
  const double* s = Sc + k * M;
  float* p = Pc + k * M;
  if (k >= n_data) {
    for (int m = lane; m < M; m += 32) p[m] = 0.f;
    return;
  }
  double mx = -INFINITY;
  for (int m = lane; m < M; m += 32) mx = fmax(mx, s[m]);
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  double sum = 0.0;
  for (int m = lane; m < M; m += 32) sum += (double)__expf((float)(s[m] - mx));
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const double lse = mx + log(sum);
  if (!isfinite(lse)) set_status(status, EMC_ERR_NUMERIC);
  for (int m = lane; m < M; m += 32) p[m] = __expf((float)(s[m] - lse));
  if (lane == 0) lse_c[k] = lse - (shift ? shift[k] : 0.0);
}

// One CTA per rotation row: Num_j = sum over the row's list of P_jk K_k; the
// K column of ones at n_pix gives den_j. Each thread owns 8 consecutive pixels
// (one 16-byte load of a K row per pair), the list is staged in shared memory
// in segments and walked four pairs at a time. Rows without pairs are zeroed.
// Poisson-fluence model (Bsum != NULL): the pairs carry P_jk B_j / N_k and
// den_j = sum P_jk is summed from the staged pairs instead.
template <bool KF16>
__global__ void __launch_bounds__(256)
    sparse_update_kernel(const uint16_t* __restrict__ Kb, int64_t ld_pix, int64_t n_pix,
                         const int64_t* __restrict__ off, const int2* __restrict__ ent, int M,
                         const float* __restrict__ Pc, float* __restrict__ Num,
                         float* __restrict__ den, const double* __restrict__ Bsum,
                         const float* __restrict__ invn) {
  const int64_t j = blockIdx.x;
  const int64_t e0 = off[j], e1 = off[j + 1];
  float* out = Num + j * ld_pix;
  constexpr int kSeg = 1024;
  __shared__ int sk[kSeg];
  __shared__ float sp[kSeg];
  __shared__ float sden[8];
  const bool flu = Bsum != nullptr;
  const float Bj = flu ? (float)Bsum[j] : 0.f;
  float dsum = 0.f;
  const int64_t n8 = ld_pix / 8;
  for (int64_t g0 = 0; g0 < n8; g0 += 256) {
    const int64_t g = g0 + threadIdx.x;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t s0 = e0; s0 < e1; s0 += kSeg) {
      const int ns = (int)min((int64_t)kSeg, e1 - s0);
      __syncthreads();
      for (int t = threadIdx.x; t < ns; t += 256) {
        const int2 km = ent[s0 + t];
        sk[t] = km.x;
        const float p = Pc[(int64_t)km.x * M + km.y];
        if (flu) {
          if (g0 == 0) dsum += p;
          sp[t] = p * (Bj * invn[km.x]);
        } else {
          sp[t] = p;
        }
      }
      __syncthreads();
      if (g < n8) {
        int t = 0;
        for (; t + 4 <= ns; t += 4) {
          uint4 w[4];
#pragma unroll
          for (int u = 0; u < 4; u++)
            w[u] = reinterpret_cast<const uint4*>(Kb + (int64_t)sk[t + u] * ld_pix)[g];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const float p = sp[t + u];
            const uint32_t wv[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
            for (int c = 0; c < 4; c++) {
              float k0, k1;
              unpack2<KF16>(wv[c], k0, k1);
              acc[2 * c] = fmaf(p, k0, acc[2 * c]);
              acc[2 * c + 1] = fmaf(p, k1, acc[2 * c + 1]);
            }
          }
        }
        for (; t < ns; t++) {
          const uint4 w = reinterpret_cast<const uint4*>(Kb + (int64_t)sk[t] * ld_pix)[g];
          const float p = sp[t];
          const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int c = 0; c < 4; c++) {
            float k0, k1;
            unpack2<KF16>(wv[c], k0, k1);
            acc[2 * c] = fmaf(p, k0, acc[2 * c]);
            acc[2 * c + 1] = fmaf(p, k1, acc[2 * c + 1]);
          }
        }
      }
    }
    if (g < n8) {
      float4* o4 = reinterpret_cast<float4*>(out + 8 * g);
      o4[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      o4[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      if (!flu && n_pix >= 8 * g && n_pix < 8 * g + 8) {
#pragma unroll
        for (int c = 0; c < 8; c++)
          if (8 * g + c == n_pix) den[j] = acc[c];
      }
    }
  }
  if (flu) {
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((threadIdx.x & 31) == 0) sden[threadIdx.x >> 5] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float d = 0.f;
      for (int w = 0; w < 8; w++) d += sden[w];
      den[j] = d;
    }
  }
}

// CSR form of the sparse update: the row Num_j accumulates in shared memory
// (FP32 atomics; a frame's non-zero pixels are distinct) from every pair's
// P_jk times the frame's non-zero counts, then is written out whole with
// den_j = sum of the row's P_jk. Rows without pairs are zeroed. Poisson-
// fluence model (Bsum != NULL): the counts are weighted by P_jk B_j / N_k.
__global__ void __launch_bounds__(256)
    sparse_update_csr_kernel(const int64_t* __restrict__ koff, const uint32_t* __restrict__ kent,
                             int64_t ld_pix, const int64_t* __restrict__ off,
                             const int2* __restrict__ ent, int M, const float* __restrict__ Pc,
                             float* __restrict__ Num, float* __restrict__ den,
                             const double* __restrict__ Bsum, const float* __restrict__ invn) {
  const int64_t j = blockIdx.x;
  const int64_t e0 = off[j], e1 = off[j + 1];
  extern __shared__ float4 sm4u[];
  float* srow = reinterpret_cast<float*>(sm4u);
  __shared__ float sden[8];
  for (int64_t i = threadIdx.x; i < ld_pix; i += blockDim.x) srow[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float dsum = 0.f;
  const float Bj = Bsum ? (float)Bsum[j] : 0.f;
  for (int64_t e = e0 + wid; e < e1; e += nw) {
    const int2 km = ent[e];
    const float p0 = Pc[(int64_t)km.x * M + km.y];
    dsum += p0;
    const float p = Bsum ? p0 * (Bj * invn[km.x]) : p0;
    const int64_t f1 = koff[km.x + 1];
    for (int64_t f = koff[km.x] + lane; f < f1; f += 32) {
      const uint32_t w = kent[f];
      atomicAdd(&srow[w & 0xffffu], p * (float)(w >> 16));
    }
  }
  if (lane == 0) sden[wid] = dsum;
  __syncthreads();
  float* out = Num + j * ld_pix;
  for (int64_t i = threadIdx.x; i < ld_pix; i += blockDim.x) out[i] = srow[i];
  if (threadIdx.x == 0) {
    float d = 0.f;
    for (int w = 0; w < nw; w++) d += sden[w];
    den[j] = d;
  }
}

// 1 - sum_{j in C_k} P_jk of a dense E-step, from its stored scores (lse2 in
// the given frame order). iperm, live (may be NULL): scores in emc_iteration's
// internal order, and the row tiles contracted there (P = 0 in the others).
__global__ void missed_mass_kernel(const float* __restrict__ S, int64_t ldS,
                                   const float* __restrict__ Sref, int64_t ld_data, const float2* __restrict__ lse2,
                                   const int32_t* __restrict__ cand, int M, int64_t n_data,
                                   const int32_t* __restrict__ iperm,
                                   const uint8_t* __restrict__ live, float* __restrict__ missed) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_data) return;
  const int64_t c = iperm ? iperm[k] : k;  // the score column
  const uint8_t* lv = live ? live + (c >> 8) : nullptr;
  const int64_t nnt = ld_data >> 8;
  const float2 L = lse2[k];
  double sum = 0.0;
  for (int m = 0; m < M; m++) {
    const int64_t j = cand[k * M + m];
    if (lv && !lv[(j >> 7) * nnt]) continue;
    const float e = S[c * ldS + j] + ((Sref[(j >> 5) * ld_data + c] - L.x) - L.y);
    sum += (double)__expf(e);
  }
  missed[k] = (float)(1.0 - sum);
}

// Responsibilities of selected frames from stored scores (Eq. 2.4):
// P[f][j] = exp(S_jk - lse_k) for k = frames[f], read like missed_mass_kernel
// (frame-major scores relative to their 32-row group maxima; iperm/live: the
// internal order and contracted tiles of a pruned pass, skipped tiles give 0).
// Grid (ceil(nrot / 256), n): threads along rotations, coalesced in S and P.
__global__ void __launch_bounds__(256)
    responsibilities_kernel(const float* __restrict__ S, int64_t ldS,
                            const float* __restrict__ Sref, int64_t ld_data,
                            const float2* __restrict__ lse2, const int32_t* __restrict__ frames,
                            int64_t nrot, int64_t n_data, const int32_t* __restrict__ iperm,
                            const uint8_t* __restrict__ live, float* __restrict__ P,
                            int32_t* status) {
  const int64_t f = blockIdx.y;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = frames[f];
  if (k < 0 || k >= n_data) {
    if (j == 0) set_status(status, EMC_ERR_ARG);
    return;
  }
  if (j >= nrot) return;
  const int64_t c = iperm ? iperm[k] : k;
  float p = 0.f;
  if (!live || live[(j >> 7) * (ld_data >> 8) + (c >> 8)]) {
    const float2 L = lse2[k];
    p = __expf(S[c * ldS + j] + ((Sref[(j >> 5) * ld_data + c] - L.x) - L.y));
  }
  P[f * nrot + j] = p;
}

// lse[k] = m_k + log s_k
__global__ void lse_values_kernel(const double* __restrict__ m, const double* __restrict__ s,
                                  int64_t n, double* __restrict__ lse) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) lse[k] = m[k] + log(s[k]);
}

cudaError_t launch_responsibilities(const float* S, int64_t ldS, const float* Sref,
                                    int64_t ld_data, const float2* lse2, const int32_t* frames,
                                    int64_t n, int64_t nrot, int64_t n_data, float* P,
                                    int32_t* status, cudaStream_t s, const int32_t* iperm,
                                    const uint8_t* live) {
  if (n <= 0) return cudaSuccess;
  dim3 grd((unsigned)((nrot + 255) / 256), (unsigned)n);
  responsibilities_kernel<<<grd, 256, 0, s>>>(S, ldS, Sref, ld_data, lse2, frames, nrot, n_data,
                                              iperm, live, P, status);
  return cudaGetLastError();
}

cudaError_t launch_lse_values(const double* m, const double* sm, int64_t n, double* lse,
                              cudaStream_t s) {
  lse_values_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, sm, n, lse);
  return cudaGetLastError();
}

cudaError_t launch_sparse_scores(const Planes& L, int precision, int64_t rows, const double* bias,
                                 const uint16_t* Kb, int64_t ld_pix, const int64_t* off,
                                 const int2* ent, int M, const int64_t* koff,
                                 const uint32_t* kent, double* Sc, cudaStream_t s) {
  const size_t smem = 2 * sizeof(float) * (size_t)ld_pix;
  cudaError_t e = cudaSuccess;
#define EMC_SPARSE_SCORES(P, C)                                                              \
  e = cudaFuncSetAttribute(sparse_scores_kernel<P, C>,                                       \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
  if (e != cudaSuccess) return e;                                                            \
  sparse_scores_kernel<P, C><<<(unsigned)rows, 256, smem, s>>>(                              \
      L.base, L.plane_stride, ld_pix, bias, Kb, off, ent, M, koff, kent, Sc)
#define EMC_SPARSE_SCORES_P(P)      \
  if (kent) {                       \
    EMC_SPARSE_SCORES(P, true);     \
  } else {                          \
    EMC_SPARSE_SCORES(P, false);    \
  }
  switch (precision) {
    case EMC_PREC_FP32: EMC_SPARSE_SCORES_P(EMC_PREC_FP32); break;
    case EMC_PREC_BF16: EMC_SPARSE_SCORES_P(EMC_PREC_BF16); break;
    case EMC_PREC_FP16_SPLIT: EMC_SPARSE_SCORES_P(EMC_PREC_FP16_SPLIT); break;
    default: EMC_SPARSE_SCORES_P(EMC_PREC_BF16_SPLIT); break;
  }
#undef EMC_SPARSE_SCORES_P
#undef EMC_SPARSE_SCORES
  return cudaGetLastError();
}

cudaError_t launch_sparse_lse(const double* Sc, int64_t n_data, int64_t ld_data, int M, float* Pc,
                              double* lse_c, int32_t* status, cudaStream_t s,
                              const double* shift) {
  sparse_lse_kernel<<<(unsigned)((ld_data * 32 + 255) / 256), 256, 0, s>>>(Sc, n_data, ld_data, M,
                                                                          Pc, lse_c, shift, status);
  return cudaGetLastError();
}

cudaError_t launch_sparse_update(const uint16_t* Kb, int kf16, int64_t ld_pix, int64_t n_pix,
                                 const int64_t* off, const int2* ent, int M, const float* Pc,
                                 int64_t rows, const int64_t* koff, const uint32_t* kent,
                                 float* Num, float* den, cudaStream_t s, const double* Bsum,
                                 const float* invn) {
  if (Bsum && !invn) return cudaErrorInvalidValue;
  if (kent) {
    const size_t smem = sizeof(float) * (size_t)ld_pix;
    cudaError_t e = cudaFuncSetAttribute(sparse_update_csr_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sparse_update_csr_kernel<<<(unsigned)rows, 256, smem, s>>>(koff, kent, ld_pix, off, ent, M, Pc,
                                                               Num, den, Bsum, invn);
    return cudaGetLastError();
  }
  if (kf16)
    sparse_update_kernel<true><<<(unsigned)rows, 256, 0, s>>>(Kb, ld_pix, n_pix, off, ent, M, Pc,
                                                              Num, den, Bsum, invn);
  else
    sparse_update_kernel<false><<<(unsigned)rows, 256, 0, s>>>(Kb, ld_pix, n_pix, off, ent, M, Pc,
                                                               Num, den, Bsum, invn);
  return cudaGetLastError();
}

cudaError_t launch_missed_mass(const float* S, int64_t ldS, const float* Sref, int64_t ld_data,
                               const float2* lse2, const int32_t* cand, int M, int64_t n_data,
                               float* missed, cudaStream_t s, const int32_t* iperm,
                               const uint8_t* live) {
  missed_mass_kernel<<<(unsigned)((n_data + 255) / 256), 256, 0, s>>>(
      S, ldS, Sref, ld_data, lse2, cand, M, n_data, iperm, live, missed);
  return cudaGetLastError();
}

}  // namespace emc
