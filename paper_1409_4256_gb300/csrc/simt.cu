// simt.cu -- FP32 SIMT form of the Maximize step (precision EMC_PREC_FP32).
//
// Scores S_jk = sum_i K_ik log W_ij + bias_j (Eq. 2.3 plus the prior of
// Eq. 2.4) as a tiled FP32 FFMA contraction over pixels: 64 rotations x 128
// frames per CTA, 4 x 8 outputs per thread, 16-pixel smem stages. Dot products
// reach |S| ~ 1e4 while P needs S to ~1e-4, beyond what a chain of FP32 FMAs
// keeps. log W is therefore split while it is staged into shared memory:
// hi = log W rounded to the 1/8 grid and r = log W - hi (|r| <= 1/16, exact).
// Counts are integers, so every partial sum of K * hi is a multiple of 1/8
// below 2^21 and the FFMA chain of the hi accumulator never rounds; the r
// accumulator stays small (a random walk of size ~ sqrt(sum K^2) / 28), so its
// rounding is ~1e-5 absolute. The epilogue adds hi + r + bias in FP64.
//  pass 1 : per frame, per tile of 64 rotations, (max_j S_jk, sum_j exp(S_jk - max))
//  pass 2 : P_jk = exp(S_jk - lse_k) written as FP32 [rows][ld_data]
//  update : Num_ji = sum_k P_jk K_ki (Eq. 2.11), FP32 FFMA; the K column of
//           ones at i = n_pix yields den_j = sum_k P_jk.
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

constexpr int SB_M = 64, SB_N = 128, SB_K = 16, S_THREADS = 256;
constexpr int SA_LD = SB_M + 4, SBN_LD = SB_N + 4;
struct ScoreAcc {
  float hi[4][8], r[4][8];
};

// Main loop shared by pass 1 and pass 2. Tile origin: rows r0, frames c0.
__device__ __forceinline__ void simt_scores_tile(const float* __restrict__ L, int64_t ld_pix,
                                                 const uint16_t* __restrict__ Kb, int64_t r0,
                                                 int64_t c0, float (*Ah)[SA_LD],
                                                 float (*Ar)[SA_LD], float (*Bs)[SBN_LD],
                                                 ScoreAcc& out) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 8; b++) {
      out.hi[a][b] = 0.f;
      out.r[a][b] = 0.f;
    }
  const int ar = t >> 2, ac = (t & 3) * 4;  // A: row, pixel offset
  const int br = t >> 1, bc = (t & 1) * 8;  // B: frame, pixel offset
  const float* Ap = L + (r0 + ar) * ld_pix + ac;
  const uint16_t* Bp = Kb + (c0 + br) * ld_pix + bc;
  const int64_t ntiles = ld_pix / SB_K;
  float4 ra = *reinterpret_cast<const float4*>(Ap);
  uint4 rb = *reinterpret_cast<const uint4*>(Bp);
  for (int64_t kt = 0; kt < ntiles; kt++) {
    __syncthreads();
    const float av4[4] = {ra.x, ra.y, ra.z, ra.w};
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const float h = rintf(av4[c] * 8.f) * 0.125f;
      Ah[ac + c][ar] = h;
      Ar[ac + c][ar] = av4[c] - h;
    }
    const uint32_t w4[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int c = 0; c < 4; c++) {
      Bs[bc + 2 * c][br] = __uint_as_float(w4[c] << 16);
      Bs[bc + 2 * c + 1][br] = __uint_as_float(w4[c] & 0xffff0000u);
    }
    __syncthreads();
    if (kt + 1 < ntiles) {
      ra = *reinterpret_cast<const float4*>(Ap + (kt + 1) * SB_K);
      rb = *reinterpret_cast<const uint4*>(Bp + (kt + 1) * SB_K);
    }
#pragma unroll
    for (int kk = 0; kk < SB_K; kk++) {
      float4 a = *reinterpret_cast<const float4*>(&Ah[kk][ty * 4]);
      float4 e = *reinterpret_cast<const float4*>(&Ar[kk][ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
      const float ah[4] = {a.x, a.y, a.z, a.w};
      const float aq[4] = {e.x, e.y, e.z, e.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) {
          out.hi[i][j] = fmaf(ah[i], bv[j], out.hi[i][j]);
          out.r[i][j] = fmaf(aq[i], bv[j], out.r[i][j]);
        }
    }
  }
}

__global__ void __launch_bounds__(S_THREADS)
    simt_pass1_kernel(const float* __restrict__ L, int64_t ld_pix, const double* __restrict__ bias,
                      const uint16_t* __restrict__ Kb, int64_t ld_data,
                      double* __restrict__ part_m, float* __restrict__ part_s,
                      float* __restrict__ S, float* __restrict__ Sref, int64_t rows) {
  __shared__ __align__(16) float Ah[SB_K][SA_LD];
  __shared__ __align__(16) float Ar[SB_K][SA_LD];
  __shared__ __align__(16) float Bs[SB_K][SBN_LD];
  __shared__ double red[16][SB_N];
  const int64_t r0 = (int64_t)blockIdx.y * SB_M, c0 = (int64_t)blockIdx.x * SB_N;
  ScoreAcc sc;
  simt_scores_tile(L, ld_pix, Kb, r0, c0, Ah, Ar, Bs, sc);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double b[4];
#pragma unroll
  for (int i = 0; i < 4; i++) b[i] = bias[r0 + ty * 4 + i];
  double x[4][8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    double m = -INFINITY;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      x[i][j] = ((double)sc.hi[i][j] + (double)sc.r[i][j]) + b[i];
      m = fmax(m, x[i][j]);
    }
    red[ty][tx * 8 + j] = m;
  }
  __syncthreads();
  double mcol[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    double m = -INFINITY;
    for (int r = 0; r < 16; r++) m = fmax(m, red[r][tx * 8 + j]);
    mcol[j] = m;
  }
  __syncthreads();
  if (S) {
    // scores relative to the tile's column maximum rounded to the 1/64 grid
    float ref[8];
#pragma unroll
    for (int j = 0; j < 8; j++)
      ref[j] = mcol[j] == -INFINITY ? -3.0e38f : (float)(rint(mcol[j] * kGridD) / kGridD);
    // frame-major: 4 consecutive rows of one column per float4
#pragma unroll
    for (int j = 0; j < 8; j++) {
      float4 v;
      v.x = (float)(x[0][j] - (double)ref[j]);
      v.y = (float)(x[1][j] - (double)ref[j]);
      v.z = (float)(x[2][j] - (double)ref[j]);
      v.w = (float)(x[3][j] - (double)ref[j]);
      *reinterpret_cast<float4*>(S + (c0 + tx * 8 + j) * rows + r0 + ty * 4) = v;
    }
    if (ty == 0) {
#pragma unroll
      for (int j = 0; j < 8; j++) {
        Sref[(r0 / 32) * ld_data + c0 + tx * 8 + j] = ref[j];
        Sref[(r0 / 32 + 1) * ld_data + c0 + tx * 8 + j] = ref[j];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 8; j++) {
    float s = 0.f;
    if (mcol[j] != -INFINITY)
#pragma unroll
      for (int i = 0; i < 4; i++) s += expf((float)(x[i][j] - mcol[j]));
    red[ty][tx * 8 + j] = (double)s;
  }
  __syncthreads();
  // threads of the first rotation group write the tile's 8 columns each
  if (ty == 0) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      double s = 0.0;
      for (int r = 0; r < 16; r++) s += red[r][tx * 8 + j];
      int64_t col = c0 + tx * 8 + j;
      part_m[(int64_t)blockIdx.y * ld_data + col] = mcol[j];
      part_s[(int64_t)blockIdx.y * ld_data + col] = (float)s;
    }
  }
}

__global__ void __launch_bounds__(S_THREADS)
    simt_normalize_kernel(const float* __restrict__ L, int64_t ld_pix,
                          const double* __restrict__ bias, int64_t nrot,
                          const uint16_t* __restrict__ Kb, int64_t ld_data, int64_t n_data,
                          const double* __restrict__ lse_m, const double* __restrict__ lse_s,
                          float* __restrict__ P) {
  __shared__ __align__(16) float Ah[SB_K][SA_LD];
  __shared__ __align__(16) float Ar[SB_K][SA_LD];
  __shared__ __align__(16) float Bs[SB_K][SBN_LD];
  const int64_t r0 = (int64_t)blockIdx.y * SB_M, c0 = (int64_t)blockIdx.x * SB_N;
  ScoreAcc sc;
  simt_scores_tile(L, ld_pix, Kb, r0, c0, Ah, Ar, Bs, sc);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double lse[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    int64_t col = c0 + tx * 8 + j;
    lse[j] = col < n_data ? lse_m[col] + log(lse_s[col]) : INFINITY;
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    int64_t row = r0 + ty * 4 + i;
    double b = bias[row];
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      double x = ((double)sc.hi[i][j] + (double)sc.r[i][j]) + b - lse[j];
      v[j] = (row < nrot && c0 + tx * 8 + j < n_data) ? expf((float)x) : 0.f;
    }
    float4* dst = reinterpret_cast<float4*>(P + row * ld_data + c0 + tx * 8);
    dst[0] = make_float4(v[0], v[1], v[2], v[3]);
    dst[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

__global__ void __launch_bounds__(S_THREADS)
    simt_update_kernel(const float* __restrict__ P, int64_t ld_data,
                       const uint16_t* __restrict__ Kb, int64_t ld_pix, int64_t n_pix,
                       float* __restrict__ Num, float* __restrict__ den) {
  __shared__ __align__(16) float As[SB_K][SA_LD];
  __shared__ __align__(16) float Bs[SB_K][SBN_LD];
  const int64_t r0 = (int64_t)blockIdx.y * SB_M, c0 = (int64_t)blockIdx.x * SB_N;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 8; b++) acc[a][b] = 0.f;
  const int ar = t >> 2, ac = (t & 3) * 4;    // A = P: row, frame offset
  const int br = t >> 4, bc = (t & 15) * 8;   // B = K: frame, pixel offset
  const bool bval = c0 + bc < ld_pix;
  const float* Ap = P + (r0 + ar) * ld_data + ac;
  const uint16_t* Bp = Kb + (int64_t)br * ld_pix + c0 + bc;
  const int64_t ntiles = ld_data / SB_K;
  float4 ra = *reinterpret_cast<const float4*>(Ap);
  uint4 rb = bval ? *reinterpret_cast<const uint4*>(Bp) : make_uint4(0, 0, 0, 0);
  for (int64_t kt = 0; kt < ntiles; kt++) {
    __syncthreads();
    As[ac + 0][ar] = ra.x;
    As[ac + 1][ar] = ra.y;
    As[ac + 2][ar] = ra.z;
    As[ac + 3][ar] = ra.w;
    const uint32_t w4[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int c = 0; c < 4; c++) {
      Bs[br][bc + 2 * c] = __uint_as_float(w4[c] << 16);
      Bs[br][bc + 2 * c + 1] = __uint_as_float(w4[c] & 0xffff0000u);
    }
    __syncthreads();
    if (kt + 1 < ntiles) {
      ra = *reinterpret_cast<const float4*>(Ap + (kt + 1) * SB_K);
      if (bval) rb = *reinterpret_cast<const uint4*>(Bp + (kt + 1) * SB_K * ld_pix);
    }
#pragma unroll
    for (int kk = 0; kk < SB_K; kk++) {
      float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    int64_t row = r0 + ty * 4 + i;
    int64_t col = c0 + tx * 8;
    if (col < ld_pix) {
      float4* dst = reinterpret_cast<float4*>(Num + row * ld_pix + col);
      dst[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      dst[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
#pragma unroll
    for (int j = 0; j < 8; j++)
      if (col + j == n_pix) den[row] = acc[i][j];
  }
}

int64_t simt_pass1_tiles(int64_t rows) { return rows / SB_M; }

cudaError_t launch_simt_pass1(const float* L, int64_t ld_pix, const double* bias, int64_t rows,
                              const uint16_t* Kb, int64_t ld_data, int64_t n_data,
                              double* part_m, float* part_s, float* S, float* Sref,
                              cudaStream_t s) {
  (void)n_data;
  dim3 grd((unsigned)(ld_data / SB_N), (unsigned)(rows / SB_M));
  simt_pass1_kernel<<<grd, S_THREADS, 0, s>>>(L, ld_pix, bias, Kb, ld_data, part_m, part_s, S,
                                              Sref, rows);
  return cudaGetLastError();
}

cudaError_t launch_simt_normalize(const float* L, int64_t ld_pix, const double* bias, int64_t rows,
                                  int64_t nrot, const uint16_t* Kb, int64_t ld_data,
                                  int64_t n_data, const double* lse_m, const double* lse_s,
                                  float* P, cudaStream_t s) {
  dim3 grd((unsigned)(ld_data / SB_N), (unsigned)(rows / SB_M));
  simt_normalize_kernel<<<grd, S_THREADS, 0, s>>>(L, ld_pix, bias, nrot, Kb, ld_data, n_data,
                                                  lse_m, lse_s, P);
  return cudaGetLastError();
}

cudaError_t launch_simt_update(const float* P, int64_t ld_data, int64_t rows, const uint16_t* Kb,
                               int64_t ld_pix, int64_t n_pix, float* Num, float* den,
                               cudaStream_t s) {
  dim3 grd((unsigned)((ld_pix + SB_N - 1) / SB_N), (unsigned)(rows / SB_M));
  simt_update_kernel<<<grd, S_THREADS, 0, s>>>(P, ld_data, Kb, ld_pix, n_pix, Num, den);
  return cudaGetLastError();
}

}  // namespace emc
