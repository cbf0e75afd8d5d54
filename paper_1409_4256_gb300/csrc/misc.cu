// misc.cu -- frame preparation, log-sum-exp merges and the final division.
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

// Frames K (Sec. 2.1) int32 [n_data][ld_k] -> BF16 (or FP16) [ld_data][ld_pix]:
// columns < n_pix hold the counts, column n_pix holds 1 for every real frame
// (so that the M-step contraction also yields den_j = sum_k P_jk), everything
// else 0. Counts outside [0, 256] (BF16; [0, 2048] FP16) or a frame total at or
// above 65536 (8192 for FP16) would break the exact conversion or the exact
// hi-term accumulation and are flagged. fp16 is a bit set: bit 0 FP16 (else
// BF16), bit 1 no limit on the total (the Gaussian model scales its operand
// to the largest total).
__global__ void prep_frames_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                                   int64_t n_pix, int64_t ld_pix, uint16_t* __restrict__ Kb,
                                   int fp16, const int32_t* __restrict__ dup_src,
                                   const int32_t* __restrict__ dup_rank, int32_t* status) {
  const int64_t k = blockIdx.x;
  __shared__ long long red[8];
  long long tot = 0;
  int bad = 0;
  const bool wide = dup_src != nullptr;
  for (int64_t i = threadIdx.x; i < ld_pix; i += blockDim.x) {
    float v = 0.f;
    if (k < n_data) {
      if (i < n_pix) {
        int32_t c = K[k * ld_k + i];
        if (c < 0 || (!wide && c > ((fp16 & 1) ? 2048 : 256))) bad = 1;
        tot += c;
        v = (float)(wide ? min(c, kDupCount) : c);
      } else if (i == n_pix) {
        v = 1.f;
      } else if (wide && i - n_pix - 1 < kDupCols) {
        // duplicate column: the part of its source pixel's count beyond the
        // parts the source column and the lower-ranked duplicates carry
        const int d = (int)(i - n_pix - 1);
        const int32_t src = dup_src[d];
        if (src >= 0) {
          const int32_t c = K[k * ld_k + src] - kDupCount * (dup_rank[d] + 1);
          v = (float)max(0, min(c, kDupCount));
        }
      }
    }
    Kb[k * ld_pix + i] = (fp16 & 1) ? fp16_bits(v) : bf16_bits(v);
  }
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    if (!(fp16 & 2) && s >= ((fp16 & 1) ? 8192 : 65536)) bad = 1;
  }
  if (bad) set_status(status, EMC_ERR_UNSUPPORTED);
}

cudaError_t launch_prep_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                               int64_t ld_data, int64_t ld_pix, uint16_t* Kb, int fp16,
                               const int32_t* dup_src, const int32_t* dup_rank,
                               int32_t* status, cudaStream_t s) {
  prep_frames_kernel<<<(unsigned)ld_data, 256, 0, s>>>(K, ld_k, n_data, n_pix, ld_pix, Kb, fp16,
                                                       dup_src, dup_rank, status);
  return cudaGetLastError();
}

// largest count of every pixel over the frames, where it exceeds kDupCount
__global__ void pixel_max_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                                 int64_t n_pix, int32_t* __restrict__ pixmax) {
  const int64_t k = blockIdx.x;
  if (k >= n_data) return;
  for (int64_t i = threadIdx.x; i < n_pix; i += blockDim.x) {
    const int32_t c = K[k * ld_k + i];
    if (c > kDupCount) atomicMax(&pixmax[i], c);
  }
}

// One thread, pixels in order: ceil(max / kDupCount) - 1 duplicate columns
// per pixel, geometry copied with w = kDupMark; unused columns reset.
__global__ void assign_duplicates_kernel(const int32_t* __restrict__ pixmax, int64_t n_pix,
                                         float4* qh, float4* ql, int16_t* fbin,
                                         int32_t* dup_src, int32_t* dup_rank, int32_t* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int nd = 0;
  for (int64_t i = 0; i < n_pix; i++) {
    const int32_t m = pixmax[i];
    if (m <= kDupCount) continue;
    const int need = (m - 1) / kDupCount;
    for (int t = 0; t < need; t++) {
      if (nd >= kDupCols) {
        set_status(status, EMC_ERR_UNSUPPORTED);
        break;
      }
      const int64_t col = n_pix + 1 + nd;
      const float4 a = qh[i];
      qh[col] = make_float4(a.x, a.y, a.z, kDupMark);
      ql[col] = ql[i];
      fbin[col] = fbin[i];
      dup_src[nd] = (int32_t)i;
      dup_rank[nd] = t;
      nd++;
    }
  }
  for (; nd < kDupCols; nd++) {
    const int64_t col = n_pix + 1 + nd;
    qh[col] = make_float4(0.f, 0.f, 0.f, 0.f);
    ql[col] = make_float4(0.f, 0.f, 0.f, 0.f);
    fbin[col] = 0;
    dup_src[nd] = -1;
    dup_rank[nd] = 0;
  }
}

cudaError_t launch_assign_duplicates(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                     int64_t ld_data, int32_t* pixmax, float4* qh, float4* ql,
                                     int16_t* fbin, int32_t* dup_src, int32_t* dup_rank,
                                     int32_t* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pixmax, 0, sizeof(int32_t) * n_pix, s);
  if (e != cudaSuccess) return e;
  pixel_max_kernel<<<(unsigned)ld_data, 256, 0, s>>>(K, ld_k, n_data, n_pix, pixmax);
  assign_duplicates_kernel<<<1, 32, 0, s>>>(pixmax, n_pix, qh, ql, fbin, dup_src, dup_rank,
                                            status);
  return cudaGetLastError();
}

// Gaussian model, per frame k: A_k = sum_i K_ik^2 and the constants the
// kernels need, gk[k] = (c_k hi, c_k lo, 2 sigma^2 / A_k, 0) with
// c_k = 1 / (2 sigma^2 A_k) split into two FP32 (0 for an empty or padding
// frame: its score is -B_j / (2 sigma^2) whatever the fluence); the largest
// frame total goes to *nmax (atomic maximum; zeroed by the caller).
__global__ void gauss_frames_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                                    int64_t n_pix, double inv2s2, float4* __restrict__ gk,
                                    unsigned long long* nmax) {
  const int64_t k = blockIdx.x;
  __shared__ long long ra[8], rn[8];
  long long a = 0, n = 0;
  if (k < n_data) {
    for (int64_t i = threadIdx.x; i < n_pix; i += blockDim.x) {
      const long long c = K[k * ld_k + i];
      a += c * c;
      n += c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rn[threadIdx.x >> 5] = n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long A = 0, Nk = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      A += ra[w];
      Nk += rn[w];
    }
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (A > 0) {
      const double c = inv2s2 / (double)A;
      const float ch = (float)c;
      g = make_float4(ch, (float)(c - (double)ch), (float)(1.0 / (inv2s2 * (double)A)), 0.f);
    }
    gk[k] = g;
    if (Nk > 0) atomicMax(nmax, (unsigned long long)Nk);
  }
}

cudaError_t launch_gauss_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                int64_t ld_data, double sigma, float4* gk,
                                unsigned long long* nmax, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(nmax, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  gauss_frames_kernel<<<(unsigned)ld_data, 256, 0, s>>>(K, ld_k, n_data, n_pix,
                                                        1.0 / (2.0 * sigma * sigma), gk, nmax);
  return cudaGetLastError();
}

// Poisson-fluence model, per frame k: N_k = sum_i K_ik, the score shift
// cn[k] = c N_k (exact in FP64: c on the 1/8 grid, N_k an integer) and
// invn[k] = 1 / N_k (0 for an empty or padding frame).
__global__ void flu_frames_kernel(const int32_t* __restrict__ K, int64_t ld_k, int64_t n_data,
                                  int64_t n_pix, double c, double* __restrict__ cn,
                                  float* __restrict__ invn) {
  const int64_t k = blockIdx.x;
  __shared__ long long rn[8];
  long long n = 0;
  if (k < n_data)
    for (int64_t i = threadIdx.x; i < n_pix; i += blockDim.x) n += K[k * ld_k + i];
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) rn[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long Nk = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) Nk += rn[w];
    cn[k] = c * (double)Nk;
    invn[k] = Nk > 0 ? (float)(1.0 / (double)Nk) : 0.f;
  }
}

cudaError_t launch_flu_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                              int64_t ld_data, double c, double* cn, float* invn,
                              cudaStream_t s) {
  flu_frames_kernel<<<(unsigned)ld_data, 256, 0, s>>>(K, ld_k, n_data, n_pix, c, cn, invn);
  return cudaGetLastError();
}

// Largest grid value (for the Gaussian scales). Non-negative floats order
// like their bit patterns, so an integer atomic maximum suffices; a
// non-finite voxel counts as +inf.
__global__ void grid_max_kernel(const float* __restrict__ grid, int64_t n, unsigned* out) {
  unsigned m = 0u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = grid[i];
    const unsigned b = isfinite(v) ? __float_as_uint(fmaxf(v, 0.f)) : 0x7f800000u;
    m = b > m ? b : m;
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void gauss_scales_kernel(const unsigned* gmax, const unsigned long long* nmax,
                                    float4* gsc, int32_t* status) {
  const float w = __uint_as_float(*gmax);
  if (!isfinite(w)) set_status(status, EMC_ERR_NUMERIC);
  *gsc = gauss_scales(w, (long long)*nmax);
}

// scratch: 16 bytes for the maximum, then the float4 scales at gsc
cudaError_t launch_gauss_scales(const float* grid, int64_t n_vox, unsigned* gmax,
                                const unsigned long long* nmax, float4* gsc, int32_t* status,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(gmax, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n_vox + 255) / 256;
  blocks = blocks < 1024 ? blocks : 1024;
  grid_max_kernel<<<(unsigned)blocks, 256, 0, s>>>(grid, n_vox, gmax);
  gauss_scales_kernel<<<1, 1, 0, s>>>(gmax, nmax, gsc, status);
  return cudaGetLastError();
}

// Per frame k: fold the per-tile pairs (m_t, s_t) -- each meaning
// sum over the tile's rotations of exp(S_jk) = s_t exp(m_t) -- into the running
// (m_k, s_k) in FP64 (Eq. 2.4's denominator; only maxima and sums travel, as
// in Sec. 3.3). Reads are coalesced along k. shift (may be NULL): a per-frame
// constant the tiles' scores carry (the Poisson-fluence model's c N_k),
// subtracted from their maxima before the merge. live (may be NULL): only row
// tiles t with live[t * nnt + k / 256] were contracted (the others underflow);
// best (may be NULL) receives the row tile of the largest maximum.
__global__ void __launch_bounds__(256)
    lse_merge_kernel(const double* __restrict__ part_m, const float* __restrict__ part_s,
                     int64_t n_tiles, int64_t ld_data, int64_t n_data, double* __restrict__ lse_m,
                     double* __restrict__ lse_s, int accumulate, double clamp,
                     const double* __restrict__ shift, const uint8_t* __restrict__ live,
                     int64_t nnt, int32_t* __restrict__ best, int32_t* status,
                     float* __restrict__ Ub, double* __restrict__ Mk, float* __restrict__ Ua) {
  // 32 frames (lanes) x 8 strides of tiles (warps); partials combined in stride order
  __shared__ double rm[8][32], rs[8][32];
  __shared__ int rb[8][32];
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * 32 + lane;
  const bool ok = k < n_data;
  const double sh = (ok && shift) ? shift[k] : 0.0;
  const uint8_t* lv = live ? live + (k >> 8) : nullptr;
  double mt = -INFINITY;
  int tbest = 0;
  // (unrolled: the flag and score loads of several tiles in flight)
  if (ok)
#pragma unroll 4
    for (int64_t t = r; t < n_tiles; t += 8) {
      if (lv && !lv[t * nnt]) continue;
      const double pmv = part_m[t * ld_data + k];
      // the tile's scores lie within 1/128 of its maximum on the 1/64 grid
      if (Ub) {
        Ub[t * ld_data + k] = __double2float_ru(pmv + 1.0 / 64.0);
        Ua[t * ld_data + k] = 0.f;
      }
      const double m = pmv - sh;
      if (m > mt) {
        mt = m;
        tbest = (int)t;
      }
    }
  rm[r][lane] = mt;
  rb[r][lane] = tbest;
  __syncthreads();
  // the largest maximum; ties go to the lowest tile, as a scan in tile order would
  mt = rm[0][lane];
  tbest = rb[0][lane];
  for (int q = 1; q < 8; q++)
    if (rm[q][lane] > mt || (rm[q][lane] == mt && rb[q][lane] < tbest)) {
      mt = rm[q][lane];
      tbest = rb[q][lane];
    }
  const double M = (ok && accumulate) ? lse_m[k] : -INFINITY;
  const double S = (ok && accumulate) ? lse_s[k] : 0.0;
  const double Mn = fmax(M, mt);
  // FP64 accumulation; the factors exp(m_t - Mn) <= 1 are taken in FP32 (relative
  // error ~1e-6 for the terms that matter, |m_t - Mn| < 30) -- FP64 exp is rare on
  // this part and the loop runs over every rotation tile
  double acc = 0.0;
  if (ok && Mn != -INFINITY)
#pragma unroll 4
    for (int64_t t = r; t < n_tiles; t += 8) {
      if (lv && !lv[t * nnt]) continue;
      const double m = part_m[t * ld_data + k] - sh;
      const float sv = part_s[t * ld_data + k];
      if (sv > 0.f) acc += (double)(sv * __expf((float)(m - Mn)));
    }
  rs[r][lane] = acc;
  __syncthreads();
  if (r != 0 || !ok) return;
  if (best) best[k] = tbest;
  if (Mk) Mk[k] = mt + sh;
  if (Mn == -INFINITY) {  // nothing seen yet
    lse_m[k] = M;
    lse_s[k] = S;
    return;
  }
  acc = (S > 0.0) ? S * exp(M - Mn) : 0.0;
  for (int q = 0; q < 8; q++) acc += rs[q][lane];
  // a best score at the clamp (Gaussian model) means every rotation was clamped
  if (!isfinite(Mn) || !(acc > 0.0) || !isfinite(acc) || Mn <= clamp)
    set_status(status, EMC_ERR_NUMERIC);
  lse_m[k] = Mn;
  lse_s[k] = acc;
}

cudaError_t launch_lse_merge(const double* part_m, const float* part_s, int64_t n_tiles,
                             int64_t ld_data, int64_t n_data, double* lse_m, double* lse_s,
                             int accumulate, int gauss, int32_t* status, cudaStream_t s,
                             const double* shift, const uint8_t* live, int32_t* best, float* Ub,
                             double* Mk, float* Ua) {
  unsigned blocks = (unsigned)((n_data + 31) / 32);
  lse_merge_kernel<<<blocks, 256, 0, s>>>(part_m, part_s, n_tiles, ld_data, n_data, lse_m, lse_s,
                                          accumulate, gauss ? -(double)kGaussClamp : -INFINITY,
                                          shift, live, ld_data / 256, best, status, Ub, Mk, Ua);
  return cudaGetLastError();
}

// Total log-likelihood sum_k (m_k + log s_k) in FP64 (lse_s NULL: sum_k m_k): one frame per thread,
// block sums combined with FP64 atomics into *out (zeroed first).
__global__ void loglik_sum_kernel(const double* __restrict__ lse_m, const double* __restrict__ lse_s,
                                  int64_t n_data, double* out) {
  __shared__ double red[8];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = k < n_data ? lse_m[k] + (lse_s ? log(lse_s[k]) : 0.0) : 0.0;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    atomicAdd(out, s);
  }
}

cudaError_t launch_loglik_sum(const double* lse_m, const double* lse_s, int64_t n_data,
                              double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  loglik_sum_kernel<<<(unsigned)((n_data + 255) / 256), 256, 0, s>>>(lse_m, lse_s, n_data, out);
  return cudaGetLastError();
}

// lse_k = m_k + log s_k (FP64) split into a part on the 1/64 grid and a small
// FP32 rest, so that kernels can subtract it from grid-aligned scores exactly.
// shift (may be NULL): the per-frame constant the scores carry, added back.
__global__ void lse_split_kernel(const double* __restrict__ lse_m, const double* __restrict__ lse_s,
                                 int64_t n_data, int64_t ld_data, const double* __restrict__ shift,
                                 float2* __restrict__ out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ld_data) return;
  if (k >= n_data) {
    out[k] = make_float2(0.f, 0.f);
    return;
  }
  const double l = lse_m[k] + log(lse_s[k]) + (shift ? shift[k] : 0.0);
  const double h = rint(l * kGridD) / kGridD;
  out[k] = make_float2((float)h, (float)(l - h));
}

cudaError_t launch_lse_split(const double* lse_m, const double* lse_s, int64_t n_data,
                             int64_t ld_data, float2* out, cudaStream_t s, const double* shift) {
  lse_split_kernel<<<(unsigned)((ld_data + 255) / 256), 256, 0, s>>>(lse_m, lse_s, n_data, ld_data,
                                                                   shift, out);
  return cudaGetLastError();
}

// E-step pass 2 from stored scores (Eq. 2.4): P_jk = exp(S_jk - lse_k) with
// S_jk held frame-major as d[k][j] (ld = ldS) relative to its 32-row group
// maximum r[j/32][k], which lies on the 1/64 grid; r - hi(lse_k) is exact, so
//   P_jk = exp(d_kj + ((r_gk - hi_k) - lo_k)).
// One CTA per 128 rows x 64 frames: every thread has eight 16-byte loads of d
// in flight (512 contiguous bytes per warp and frame), the tile is transposed
// through shared memory with its columns XOR-swizzled by 4 (k / 8 mod 8), so
// that the reads along k are free of bank conflicts, and P is written along k
// (128 contiguous bytes per row and plane). The lse split and the group maxima
// of the tile are staged in shared memory. HBM-bound: 4 B read and 4 B written
// per (j, k).
//
// Gaussian model (OUT 4): after P, the M-step operand of Eq. 2.5 with the
// fluence of Eq. 2.6, P_jk / phi_jk, where
//   1/phi_jk = G_jk / A_k = sqrt((S_jk - bias_j) 2 sigma^2 / A_k)
// and S_jk - bias_j = G_jk^2 / (2 sigma^2 A_k) >= 0 is formed as
// d + (r - hi(bias_j)) - lo(bias_j) (r and hi(bias) on the 1/64 grid, so the
// large parts cancel exactly). Written as BF16 hi + lo (relative precision
// 2^-17 over the whole FP32 range, which a single FP16 scale cannot give rows
// of small responsibility); den_j = sum_k P_jk is added to den with one FP32
// atomic per row and 8 frames (den zeroed by the caller).
//
// Poisson-fluence model (OUT 5): the M-step operand P_jk / phi_jk =
// P_jk B_j / N_k in BF16 hi + lo (0 for an empty frame) and den_j as for OUT 4.
struct NormArgs {
  const float* S;
  int64_t ldS;
  const float* Sref;
  const float2* lse2;
  int64_t nrot, ld_data, n_data;
  void* P;
  int64_t P_plane;
  const double* bias;  // Gaussian
  const float4* gk;    // Gaussian: .z = 2 sigma^2 / A_k
  float* den;          // Gaussian, Poisson-fluence
  const double* Bsum;  // Poisson-fluence: B_j
  const float* invn;   // Poisson-fluence: 1 / N_k
  uint8_t* kb_flag;    // optional: 1 where the CTA's 128 x 64 block of P is non-zero;
                       // blocks found zero are then not written (their readers skip them)
  int64_t kb_ld;
  const uint8_t* tile_live;  // optional: [row tile][256-frame tile] of a pruned pass 1;
                             // a block in a tile not contracted has P = 0
};

// A 32-row group of stored scores whose maximum r lies more than 110 below
// lse_k has P_jk = exp(d + r - lse_k) = 0 exactly for all its rows (d <= 2^-7,
// and e^-110 < 2^-158 is below FP32's smallest subnormal, however exp is
// evaluated): such groups are not read.
constexpr float kUnderflowArg = -110.0f;

constexpr int kNormRows = 128, kNormFrames = 64;

// OUT: 0 FP32 P; 1 BF16 hi plane only; 2 BF16 hi + lo; 3 FP16 hi + lo of 2^14 P;
// 4 Gaussian BF16 hi + lo of P / phi plus den; 5 Poisson-fluence, likewise
template <int OUT>
__global__ void __launch_bounds__(256) normalize_scores_kernel(const NormArgs a) {
  __shared__ __align__(16) float tile[kNormFrames][kNormRows];
  __shared__ float2 sl[kNormFrames];
  __shared__ float sr[kNormRows / 32][kNormFrames];
  __shared__ float sg[kNormFrames];
  const int64_t j0 = (int64_t)blockIdx.y * kNormRows, k0 = (int64_t)blockIdx.x * kNormFrames;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kNormFrames) {
    sl[tid] = a.lse2[k0 + tid];
    if (OUT == 4) sg[tid] = a.gk[k0 + tid].z;
    if (OUT == 5) sg[tid] = a.invn[k0 + tid];
  }
  sr[tid >> 6][tid & 63] = a.Sref[((j0 >> 5) + (tid >> 6)) * a.ld_data + k0 + (tid & 63)];
  __syncthreads();
  {  // a block whose every (group, frame) underflows: P = 0 without reading S
    const int gk = tid & 63;
    const bool tile_on =
        !a.tile_live || a.tile_live[(int64_t)blockIdx.y * (a.ld_data >> 8) + (k0 >> 8)];
    const bool live = tile_on && (sr[tid >> 6][gk] - sl[gk].x) - sl[gk].y >= kUnderflowArg;
    if (!__syncthreads_or(live)) {
      if (a.kb_flag) {
        if (tid == 0) a.kb_flag[(int64_t)blockIdx.y * a.kb_ld + blockIdx.x] = 0;
        return;
      }
      // dense output: zeros, 32 frames of one row per thread
      const int64_t j = j0 + (tid >> 1), k = k0 + 32 * (tid & 1);
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      if (OUT == 0) {
        uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<float*>(a.P) + j * a.ld_data + k);
#pragma unroll
        for (int q = 0; q < 8; q++) o[q] = z;
      } else {
        uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(a.P) + j * a.ld_data + k);
        uint4* o2 = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(a.P) + a.P_plane +
                                             j * a.ld_data + k);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          o[q] = z;
          o2[q] = z;
        }
      }
      return;
    }
  }
  float4 v[8];
#pragma unroll
  for (int r = 0; r < 8; r++) {  // warp w: frames w + 8 r; lane: rows 4 lane .. 4 lane + 3
    const int k = warp + 8 * r;
    const float2 lk = sl[k];
    if ((sr[lane >> 3][k] - lk.x) - lk.y >= kUnderflowArg)
      v[r] = __ldcs(reinterpret_cast<const float4*>(a.S + (k0 + k) * a.ldS + j0) + lane);
    else  // the lane's 4 rows lie in an underflowing group: P = 0
      v[r] = make_float4(-1.0e30f, -1.0e30f, -1.0e30f, -1.0e30f);
  }
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const int k = warp + 8 * r;  // (k >> 3) & 7 == r
    *reinterpret_cast<float4*>(&tile[k][(4 * lane) ^ (4 * r)]) = v[r];
  }
  __syncthreads();
  const int kq = tid & 7, kb = 8 * kq, sw = 4 * kq;  // frames kb .. kb + 7
  float2 L[8];
#pragma unroll
  for (int u = 0; u < 8; u++) L[u] = sl[kb + u];
  int nz = 0;
#pragma unroll 1
  for (int pass = 0; pass < kNormRows / 32; pass++) {
    const int jj = (tid >> 3) + 32 * pass;
    const int64_t j = j0 + jj, k = k0 + kb;
    const bool row_ok = j < a.nrot;
    float bh = 0.f, bl = 0.f;
    if (OUT == 4 && row_ok) {
      const double b = a.bias[j];
      bh = (float)(rint(b * kGridD) / kGridD);
      bl = (float)(b - (double)bh);
    }
    const float Bj = (OUT == 5 && row_ok) ? (float)a.Bsum[j] : 0.f;
    float p[8], dsum = 0.f;
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const float d = tile[kb + u][jj ^ sw];
      const float r = sr[pass][kb + u];
      const bool ok = row_ok && k + u < a.n_data;
      const float pr = ok ? __expf(d + ((r - L[u].x) - L[u].y)) : 0.f;
      if (OUT == 4) {
        dsum += pr;
        const float q = fmaxf(d + ((r - bh) - bl), 0.f);
        p[u] = ok ? pr * sqrtf(q * sg[kb + u]) : 0.f;
      } else if (OUT == 5) {
        dsum += pr;
        p[u] = pr * (Bj * sg[kb + u]);
      } else {
        p[u] = pr;
      }
    }
    if (OUT == 0) {
      float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.P) + j * a.ld_data + k);
      o[0] = make_float4(p[0], p[1], p[2], p[3]);
      o[1] = make_float4(p[4], p[5], p[6], p[7]);
#pragma unroll
      for (int u = 0; u < 8; u++) nz |= p[u] != 0.f;
    } else {
      uint32_t h[4], l[4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        uint16_t h0, h1, l0, l1;
        if (OUT == 3) {
          const float s0 = p[u] * kP16Scale, s1 = p[u + 1] * kP16Scale;
          h0 = fp16_bits(s0);
          h1 = fp16_bits(s1);
          l0 = fp16_bits(s0 - fp16_val(h0));
          l1 = fp16_bits(s1 - fp16_val(h1));
        } else {
          h0 = bf16_bits(p[u]);
          h1 = bf16_bits(p[u + 1]);
          l0 = OUT != 1 ? bf16_bits(p[u] - bf16_val(h0)) : (uint16_t)0;
          l1 = OUT != 1 ? bf16_bits(p[u + 1] - bf16_val(h1)) : (uint16_t)0;
        }
        h[u / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
        l[u / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
      }
      uint16_t* ph = reinterpret_cast<uint16_t*>(a.P) + j * a.ld_data + k;
      *reinterpret_cast<uint4*>(ph) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(ph + a.P_plane) = make_uint4(l[0], l[1], l[2], l[3]);
      nz |= (h[0] | h[1] | h[2] | h[3] | l[0] | l[1] | l[2] | l[3]) != 0u;
    }
    if (OUT == 4 || OUT == 5) {  // the 8 threads of a row are consecutive lanes
      dsum += __shfl_xor_sync(0xffffffffu, dsum, 1);
      dsum += __shfl_xor_sync(0xffffffffu, dsum, 2);
      dsum += __shfl_xor_sync(0xffffffffu, dsum, 4);
      if (kq == 0 && row_ok && dsum > 0.f) atomicAdd(a.den + j, dsum);
    }
  }
  if (a.kb_flag) {  // uniform: every thread reaches the barrier
    const int any = __syncthreads_or(nz);
    if (tid == 0) a.kb_flag[(int64_t)blockIdx.y * a.kb_ld + blockIdx.x] = any ? 1 : 0;
  }
}

// rows: multiple of 128 (the stored-score blocks are); ld_data: multiple of 256
cudaError_t launch_normalize_scores(const float* S, int64_t ldS, const float* Sref,
                                    const float2* lse2, int64_t rows, int64_t nrot,
                                    int64_t ld_data, int64_t n_data, int precision, void* P,
                                    int64_t P_plane, cudaStream_t s, uint8_t* kb_flag,
                                    const uint8_t* tile_live) {
  NormArgs a{S, ldS, Sref, lse2, nrot, ld_data, n_data, P, P_plane,
             nullptr, nullptr, nullptr, nullptr, nullptr};
  a.kb_flag = kb_flag;
  a.kb_ld = ld_data / kNormFrames;
  a.tile_live = tile_live;
  dim3 grid((unsigned)(ld_data / kNormFrames), (unsigned)(rows / kNormRows));
  if (precision == EMC_PREC_FP32)
    normalize_scores_kernel<0><<<grid, 256, 0, s>>>(a);
  else if (precision == EMC_PREC_FP16_SPLIT)
    normalize_scores_kernel<3><<<grid, 256, 0, s>>>(a);
  else if (precision == EMC_PREC_BF16)
    normalize_scores_kernel<1><<<grid, 256, 0, s>>>(a);
  else
    normalize_scores_kernel<2><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_normalize_scores_gauss(const float* S, int64_t ldS, const float* Sref,
                                          const float2* lse2, const double* bias,
                                          const float4* gk, int64_t rows, int64_t nrot,
                                          int64_t ld_data, int64_t n_data, uint16_t* P,
                                          int64_t P_plane, float* den, cudaStream_t s,
                                          uint8_t* kb_flag) {
  cudaError_t e = cudaMemsetAsync(den, 0, sizeof(float) * rows, s);
  if (e != cudaSuccess) return e;
  NormArgs a{S, ldS, Sref, lse2, nrot, ld_data, n_data, P, P_plane, bias, gk, den, nullptr,
             nullptr};
  a.kb_flag = kb_flag;
  a.kb_ld = ld_data / kNormFrames;
  dim3 grid((unsigned)(ld_data / kNormFrames), (unsigned)(rows / kNormRows));
  normalize_scores_kernel<4><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_normalize_scores_flu(const float* S, int64_t ldS, const float* Sref,
                                        const float2* lse2, const double* Bsum, const float* invn,
                                        int64_t rows, int64_t nrot, int64_t ld_data,
                                        int64_t n_data, uint16_t* P, int64_t P_plane, float* den,
                                        cudaStream_t s, uint8_t* kb_flag,
                                        const uint8_t* tile_live) {
  cudaError_t e = cudaMemsetAsync(den, 0, sizeof(float) * rows, s);
  if (e != cudaSuccess) return e;
  NormArgs a{S, ldS, Sref, lse2, nrot, ld_data, n_data, P, P_plane, nullptr, nullptr, den, Bsum,
             invn};
  a.kb_flag = kb_flag;
  a.kb_ld = ld_data / kNormFrames;
  a.tile_live = tile_live;
  dim3 grid((unsigned)(ld_data / kNormFrames), (unsigned)(rows / kNormRows));
  normalize_scores_kernel<5><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// Per row tile mt (one warp each): the indices of the 64-frame blocks whose
// flag is set, in order, into list[mt * kb_ld ..] and their number into cnt[mt]
// (the update then contracts only those blocks of P).
__global__ void kb_lists_kernel(const uint8_t* __restrict__ flag, int64_t n_mtiles, int kb_ld,
                                int32_t* __restrict__ cnt, int32_t* __restrict__ list) {
  const int64_t mt = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (mt >= n_mtiles) return;
  const uint8_t* f = flag + mt * kb_ld;
  int32_t* out = list + mt * kb_ld;
  int n = 0;
  for (int b0 = 0; b0 < kb_ld; b0 += 32) {
    const bool on = b0 + lane < kb_ld && f[b0 + lane] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (on) out[n + __popc(m & ((1u << lane) - 1u))] = b0 + lane;
    n += __popc(m);
  }
  if (lane == 0) cnt[mt] = n;
}

cudaError_t launch_kb_lists(const uint8_t* flag, int64_t n_mtiles, int kb_ld, int32_t* cnt,
                            int32_t* list, cudaStream_t s) {
  const int64_t threads = n_mtiles * 32;
  kb_lists_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(flag, n_mtiles, kb_ld, cnt,
                                                                   list);
  return cudaGetLastError();
}

// Eq. 2.12's final division (the paper's insert_slices_division), over voxels.
__global__ void finalize_kernel(int64_t n_vox, const double* __restrict__ g_num,
                                const double* __restrict__ g_den, int nrep,
                                const float* grid_prev, float* grid_out) {
  int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_vox) return;
  double n = 0.0, d = 0.0;
  for (int r = 0; r < nrep; r++) {  // the compression's grid replicas
    n += g_num[r * n_vox + l];
    d += g_den[r * n_vox + l];
  }
  grid_out[l] = d > 0.0 ? (float)(n / d) : grid_prev[l];
}

cudaError_t launch_finalize(int64_t n_vox, const double* g_num, const double* g_den, int nrep,
                            const float* grid_prev, float* grid_out, cudaStream_t s) {
  unsigned blocks = (unsigned)((n_vox + 255) / 256);
  finalize_kernel<<<blocks, 256, 0, s>>>(n_vox, g_num, g_den, nrep, grid_prev, grid_out);
  return cudaGetLastError();
}

}  // namespace emc
