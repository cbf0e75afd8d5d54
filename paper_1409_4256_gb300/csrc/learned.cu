// learned.cu -- learned rotation proposal: binned frame features and a small
// MLP (512 -> 3 x 512 GELU -> one logit per rotation) with hand-written
// forward, backward and Adam kernels.
//
// The paper has no learned component; this is the workload's proposal stage:
// the network reads 32 radial x 16 angular bins of log(1 + mean count) of a
// frame and is trained on soft targets taken from dense EMC responsibilities
// (Eq. 2.4), so that the Maximize step can run over its top-M rotations only.
//
// Matrix products use BF16-rounded operands with FP32 accumulation ("BF16
// matmuls, FP32 master weights"). The output layer (512 x n_out, nearly all
// of the work) runs on the tensor cores through the update form of the
// tcgen05 kernel (K-major A, MN-major B, FP32 rows out): Z = H3 W4,
// dH3 = dZ (W4^T) and dW4 = (H3^T) dZ, from BF16 copies (W4, its transpose,
// H3^T, dZ) made by the kernels below, whenever the batch is a multiple of
// 128. The 512 x 512 layers and other batches use a tiled SIMT kernel that
// serves the three layouts (X W, dY W^T, X^T dY). Parameters live in one FP32
// array: W1[512][512] b1[512] W2 b2 W3 b3 W4[512][ld_out] b4[ld_out],
// ld_out = round_up(n_out, 64).
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

// ---------------------------------------------------------------- features --
// One CTA per frame: per-bin sums of the counts in shared memory, then
// log(1 + sum / pixels-in-bin); bins with no pixel give 0.
__global__ void features_kernel(const uint16_t* __restrict__ Kb, int kf16, int64_t ld_pix,
                                int64_t n_pix,
                                int64_t n_data, const int16_t* __restrict__ bin,
                                const float* __restrict__ inv_count, float* __restrict__ feat) {
  const int64_t k = blockIdx.x;
  __shared__ float acc[kFeat];
  for (int b = threadIdx.x; b < kFeat; b += blockDim.x) acc[b] = 0.f;
  __syncthreads();
  if (k < n_data)
    for (int64_t i = threadIdx.x; i < ld_pix; i += blockDim.x) {  // pixels + duplicate columns
      if (i == n_pix) continue;  // the column of ones
      const uint16_t u = Kb[k * ld_pix + i];
      const float c = kf16 ? fp16_val(u) : bf16_val(u);
      if (c != 0.f) atomicAdd(&acc[bin[i]], c);
    }
  __syncthreads();
  for (int b = threadIdx.x; b < kFeat; b += blockDim.x)
    feat[k * kFeat + b] = k < n_data ? log1pf(acc[b] * inv_count[b]) : 0.f;
}

cudaError_t launch_features(const uint16_t* Kb, int kf16, int64_t ld_pix, int64_t n_pix,
                            int64_t n_data, int64_t ld_data, const int16_t* bin,
                            const float* inv_count, float* feat, cudaStream_t s) {
  features_kernel<<<(unsigned)ld_data, 256, 0, s>>>(Kb, kf16, ld_pix, n_pix, n_data, bin,
                                                    inv_count, feat);
  return cudaGetLastError();
}

// -------------------------------------------------------------------- GEMM --
// C[M][N] = op(A) op(B) (+ bias[N]); op(A)[m][k] = TA ? A[k*lda + m] : A[m*lda + k],
// op(B)[k][n] = TB ? B[n*ldb + k] : B[k*ldb + n]. EPI: 0 plain, 1 bias,
// 2 bias + GELU (the pre-activation goes to `pre`, GELU of it to C).
constexpr int G_BM = 64, G_BN = 64, G_BK = 16, G_THREADS = 256;

__device__ __forceinline__ float bf16_round(float x) { return bf16_val(bf16_bits(x)); }

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) +
         x * __expf(-0.5f * x * x) * 0.39894228040143268f;
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(G_THREADS)
    mlp_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int64_t lda,
                    const float* __restrict__ B, int64_t ldb, float* __restrict__ C, int64_t ldc,
                    const float* __restrict__ bias, float* __restrict__ pre, int64_t ldpre) {
  __shared__ float As[G_BK][G_BM + 4];
  __shared__ float Bs[G_BK][G_BN + 4];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * G_BM, n0 = blockIdx.x * G_BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += G_BK) {
    // 64 x 16 tiles of op(A) and 16 x 64 of op(B): 4 elements per thread each
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int e = t + u * G_THREADS;
      {
        int mm, kk;
        if (TA) { kk = e / G_BM; mm = e % G_BM; } else { mm = e / G_BK; kk = e % G_BK; }
        const int gm = m0 + mm, gk = k0 + kk;
        float v = 0.f;
        if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
        As[kk][mm] = bf16_round(v);
      }
      {
        int nn, kk;
        if (TB) { nn = e / G_BK; kk = e % G_BK; } else { kk = e / G_BN; nn = e % G_BN; }
        const int gn = n0 + nn, gk = k0 + kk;
        float v = 0.f;
        if (gn < N && gk < K) v = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
        Bs[kk][nn] = bf16_round(v);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < G_BK; kk++) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (EPI >= 1) v += bias[gn];
      if (EPI == 2) {
        pre[(int64_t)gm * ldpre + gn] = v;
        v = gelu_f(v);
      }
      C[(int64_t)gm * ldc + gn] = v;
    }
  }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const float* A, int64_t lda, const float* B, int64_t ldb,
                 float* C, int64_t ldc, const float* bias, float* pre, int64_t ldpre,
                 cudaStream_t s) {
  dim3 grid((unsigned)((N + G_BN - 1) / G_BN), (unsigned)((M + G_BM - 1) / G_BM));
  mlp_gemm_kernel<TA, TB, EPI><<<grid, G_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias,
                                                          pre, ldpre);
  return cudaGetLastError();
}

// ------------------------------------------- BF16 operands for the tcgen05 --
__global__ void to_bf16_kernel(const float* __restrict__ src, int64_t n, uint16_t* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = bf16_bits(src[i]);
}

// dst[c][r] = bf16(src[r][c]) for r < rows, c < cols (32 x 32 tiles through
// shared memory; rows and cols multiples of 32)
__global__ void transpose_bf16_kernel(const float* __restrict__ src, int64_t ld_src, int64_t rows,
                                      int64_t cols, uint16_t* __restrict__ dst, int64_t ld_dst) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) t[k][tx] = src[(r0 + k) * ld_src + c0 + tx];
  __syncthreads();
  for (int k = ty; k < 32; k += 8) dst[(c0 + k) * ld_dst + r0 + tx] = bf16_bits(t[tx][k]);
}

__global__ void add_bias_kernel(float* __restrict__ Z, int64_t ld, int64_t rows, int64_t cols,
                                const float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows * cols) Z[(i / cols) * ld + i % cols] += b[i % cols];
}

cudaError_t to_bf16(const float* src, int64_t n, uint16_t* dst, cudaStream_t s) {
  to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, dst);
  return cudaGetLastError();
}
cudaError_t transpose_bf16(const float* src, int64_t ld_src, int64_t rows, int64_t cols,
                           uint16_t* dst, int64_t ld_dst, cudaStream_t s) {
  dim3 grid((unsigned)(cols / 32), (unsigned)(rows / 32));
  transpose_bf16_kernel<<<grid, 256, 0, s>>>(src, ld_src, rows, cols, dst, ld_dst);
  return cudaGetLastError();
}

// C[M][N] (FP32, row stride N) = A[M][K] (BF16, K contiguous) B[K][N] (BF16, N
// contiguous) on the tensor cores; M multiple of 128, K and N multiples of 64
cudaError_t tc_gemm(const uint16_t* A, int64_t M, int64_t K, const uint16_t* B, int64_t N,
                    float* C, int32_t* status, cudaStream_t s) {
  Planes pa{const_cast<uint16_t*>(A), M * K, K};
  return launch_tc_update(pa, EMC_PREC_BF16, M, B, K, N, INT64_MAX, C, nullptr, status, s);
}

// ------------------------------------------------- loss and its gradient --
// Row b of z (n_out logits, stride ld): lse = log sum_j exp(z_j); loss
// += -sum_r p_r (z_{idx_r} - lse) / B; z is overwritten by
// dL/dz = (softmax(z) sum_r p_r - onehot(p)) / B (zero beyond n_out).
__global__ void softmax_ce_kernel(float* __restrict__ z, int64_t ld, int n_out,
                                  const int32_t* __restrict__ tidx, const float* __restrict__ tprob,
                                  int R, int B, double* loss) {
  const int64_t b = blockIdx.x;
  float* row = z + b * ld;
  __shared__ float red[32];
  __shared__ double dred[32];
  __shared__ float s_lse;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float m = -INFINITY;
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) m = fmaxf(m, row[j]);
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = red[0];
    for (int w = 1; w < nw; w++) mm = fmaxf(mm, red[w]);
    red[0] = mm;
  }
  __syncthreads();
  m = red[0];
  double se = 0.0;
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) se += (double)__expf(row[j] - m);
  for (int o = 16; o; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  if (lane == 0) dred[wid] = se;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; w++) t += dred[w];
    s_lse = m + (float)log(t);
    // loss and the total target mass, before z is overwritten
    double l = 0.0;
    for (int r = 0; r < R; r++) {
      const float p = tprob[b * R + r];
      l -= (double)p * ((double)row[tidx[b * R + r]] - (double)s_lse);
    }
    atomicAdd(loss, l / B);
  }
  __syncthreads();
  const float lse = s_lse;
  float tm = 0.f;
  for (int r = 0; r < R; r++) tm += tprob[b * R + r];
  const float invB = 1.f / (float)B;
  for (int j = threadIdx.x; j < (int)ld; j += blockDim.x)
    row[j] = j < n_out ? __expf(row[j] - lse) * tm * invB : 0.f;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int r = 0; r < R; r++) row[tidx[b * R + r]] -= tprob[b * R + r] * invB;
}

// out[c] = sum_r X[r][c] (bias gradients)
__global__ void colsum_kernel(const float* __restrict__ X, int rows, int cols, int64_t ld,
                              float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; r++) s += X[(int64_t)r * ld + c];
  out[c] = s;
}

// d = g * GELU'(a), elementwise
__global__ void gelu_backward_kernel(const float* __restrict__ g, const float* __restrict__ a,
                                     float* __restrict__ d, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = g[i] * gelu_grad_f(a[i]);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ------------------------------------------------------------ host side --
MlpLayout mlp_layout(int64_t n_out, int64_t B) {
  MlpLayout y;
  y.n_out = n_out;
  y.ld_out = (n_out + 63) / 64 * 64;
  const int64_t H = kFeat;
  int64_t o = 0;
  for (int l = 0; l < 3; l++) {
    y.W[l] = o;
    o += H * H;
    y.b[l] = o;
    o += H;
  }
  y.W[3] = o;
  o += H * y.ld_out;
  y.b[3] = o;
  o += y.ld_out;
  y.n_params = o;
  // work: pre-activations a[3], activations h[3], dh, da (each B x 512), z / dz (B x ld_out),
  // then the tensor-core path's BF16 copies: H3 [B][512], H3^T [512][B], dZ [B][ld_out],
  // W4 [512][ld_out], W4^T [ld_out][512], each from a 256-byte boundary
  y.B = B;
  auto up64 = [](int64_t n) { return (n + 63) / 64 * 64; };  // floats to 256 bytes
  y.work_floats = up64(8 * B * H + B * y.ld_out) + up64(B * H / 2) + up64(B * H / 2) +
                  up64(B * y.ld_out / 2) + 2 * up64(H * y.ld_out / 2);
  return y;
}

namespace {
struct Work {
  float* a[3];
  float* h[3];
  float* dh;
  float* da;
  float* z;
  uint16_t *h3b, *h3t, *dzb, *w4b, *w4t;  // BF16 operands of the tensor-core products
};
Work carve(const MlpLayout& y, float* w) {
  Work k;
  const int64_t H = kFeat, BH = y.B * H;
  auto up64 = [](int64_t n) { return (n + 63) / 64 * 64; };
  for (int l = 0; l < 3; l++) k.a[l] = w + l * BH;
  for (int l = 0; l < 3; l++) k.h[l] = w + (3 + l) * BH;
  k.dh = w + 6 * BH;
  k.da = w + 7 * BH;
  k.z = w + 8 * BH;
  float* o = w + up64(8 * BH + y.B * y.ld_out);
  k.h3b = reinterpret_cast<uint16_t*>(o);
  o += up64(BH / 2);
  k.h3t = reinterpret_cast<uint16_t*>(o);
  o += up64(BH / 2);
  k.dzb = reinterpret_cast<uint16_t*>(o);
  o += up64(y.B * y.ld_out / 2);
  k.w4b = reinterpret_cast<uint16_t*>(o);
  o += up64(H * y.ld_out / 2);
  k.w4t = reinterpret_cast<uint16_t*>(o);
  return k;
}
bool tc_batch(int B) { return B >= 128 && B % 128 == 0; }
}  // namespace

cudaError_t mlp_forward(const MlpLayout& y, const float* params, const float* X, int B,
                        float* work, float* logits, cudaStream_t s) {
  Work w = carve(y, work);
  const int H = kFeat;
  const float* in = X;
  cudaError_t e;
  for (int l = 0; l < 3; l++) {
    e = gemm<false, false, 2>(B, H, H, in, H, params + y.W[l], H, w.h[l], H, params + y.b[l],
                              w.a[l], H, s);
    if (e != cudaSuccess) return e;
    in = w.h[l];
  }
  if (!tc_batch(B))
    return gemm<false, false, 1>(B, (int)y.n_out, H, in, H, params + y.W[3], y.ld_out, logits,
                                 y.ld_out, params + y.b[3], nullptr, 0, s);
  // output layer on the tensor cores: logits = bf16(H3) bf16(W4) + b4
  if ((e = to_bf16(in, (int64_t)B * H, w.h3b, s)) != cudaSuccess) return e;
  if ((e = to_bf16(params + y.W[3], (int64_t)H * y.ld_out, w.w4b, s)) != cudaSuccess) return e;
  if ((e = tc_gemm(w.h3b, B, H, w.w4b, y.ld_out, logits, nullptr, s)) != cudaSuccess) return e;
  const int64_t n = (int64_t)B * y.n_out;
  add_bias_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(logits, y.ld_out, B, y.n_out,
                                                            params + y.b[3]);
  return cudaGetLastError();
}

cudaError_t mlp_train_step(const MlpLayout& y, float* params, float* grads, float* adam_m,
                           float* adam_v, int step, float lr, const float* X,
                           const int32_t* tidx, const float* tprob, int B, int R, float* work,
                           double* loss, cudaStream_t s) {
  Work w = carve(y, work);
  const int H = kFeat;
  cudaError_t e = mlp_forward(y, params, X, B, work, w.z, s);
  if (e != cudaSuccess) return e;
  softmax_ce_kernel<<<B, 256, 0, s>>>(w.z, y.ld_out, (int)y.n_out, tidx, tprob, R, B, loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // output layer: dW4 = h3^T dz, db4 = colsum(dz), dh3 = dz W4^T
  const float* g = w.z;
  int64_t ldg = y.ld_out;
  int ncol = (int)y.n_out;
  for (int l = 3; l >= 0; l--) {
    const float* in = l == 0 ? X : w.h[l - 1];
    const int64_t ldw = l == 3 ? y.ld_out : H;
    const bool tc = l == 3 && tc_batch(B);
    if (tc) {
      // dW4 = bf16(H3)^T bf16(dZ) and dH3 = bf16(dZ) bf16(W4)^T on the tensor cores
      // (the whole padded width: dZ is 0 beyond n_out)
      if ((e = to_bf16(g, (int64_t)B * y.ld_out, w.dzb, s)) != cudaSuccess) return e;
      if ((e = transpose_bf16(in, H, B, H, w.h3t, B, s)) != cudaSuccess) return e;
      if ((e = tc_gemm(w.h3t, H, B, w.dzb, y.ld_out, grads + y.W[3], nullptr, s)) != cudaSuccess)
        return e;
    } else {
      e = gemm<true, false, 0>(H, ncol, B, in, H, g, ldg, grads + y.W[l], ldw, nullptr, nullptr,
                               0, s);
      if (e != cudaSuccess) return e;
    }
    colsum_kernel<<<(ncol + 255) / 256, 256, 0, s>>>(g, B, ncol, ldg, grads + y.b[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l == 0) break;
    if (tc) {
      if ((e = transpose_bf16(params + y.W[3], y.ld_out, H, y.ld_out, w.w4t, H, s)) != cudaSuccess)
        return e;
      if ((e = tc_gemm(w.dzb, B, y.ld_out, w.w4t, H, w.dh, nullptr, s)) != cudaSuccess) return e;
    } else {
      e = gemm<false, true, 0>(B, H, ncol, g, ldg, params + y.W[l], ldw, w.dh, H, nullptr,
                               nullptr, 0, s);
      if (e != cudaSuccess) return e;
    }
    const int64_t n = (int64_t)B * H;
    gelu_backward_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.dh, w.a[l - 1], w.da, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    g = w.da;
    ldg = H;
    ncol = H;
  }
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(unsigned)((y.n_params + 255) / 256), 256, 0, s>>>(params, grads, adam_m, adam_v,
                                                                  y.n_params, lr, b1, b2, 1e-8f,
                                                                  bc1, bc2);
  return cudaGetLastError();
}

}  // namespace emc
