// compress.cu -- c-step of EMC (Eq. 2.12; Eq. 2.5 + 2.10 in IDW mode).
//
// One CTA per rotation row j, threads over pixels. Each (i, j) recomputes the
// double-float grid point p = R_j q_i + N/2 (the same weights f(p_l - R_j q_i)
// that expansion used) and scatters f * Num_ij into g_num and f * den_j into
// g_den with FP64 atomics resolved in L2 (the N^3 FP64 grids, 2 MB at 64^3,
// stay L2-resident). The paper's insert_slices kernel also used one block
// per slice. Rotations without responsibility mass (den_j = 0) are skipped.
// Every slice passes through the centre of the grid, so concurrent CTAs
// reduce into the same central voxels; with nrep > 1 the CTA of row j uses
// grid replica j mod nrep (nrep x N^3 per grid, summed by the final division)
// to spread those reductions over more addresses.
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

constexpr int kCompressThreads = 256;

// INTERIOR: all trilinear corners of every pixel lie inside the grid (checked
// on the host from max |q_i|), so no bounds checks and one base index.
template <bool INTERIOR>
__global__ void __launch_bounds__(kCompressThreads)
    compress_kernel(const float4* __restrict__ qh, const float4* __restrict__ ql, int64_t n_pix,
                    int64_t ld_pix, int N, const RotDF* __restrict__ rot,
                    const float* __restrict__ Num, const float* __restrict__ den, int mode,
                    double* __restrict__ g_num, double* __restrict__ g_den, int nrep,
                    int64_t n_vox) {
  const int64_t row = blockIdx.x;
  const int64_t rep = (row % nrep) * n_vox;
  g_num += rep;
  g_den += rep;
  __shared__ RotDF R;
  const float dj = den[row];
  // a rotation without responsibility mass has Num = 0 and den = 0 (both
  // modes): it adds nothing, and sparse iterations leave most rows so
  if (!(dj > 0.f)) return;
  if (threadIdx.x < 18)
    reinterpret_cast<float*>(&R)[threadIdx.x] = reinterpret_cast<const float*>(rot + row)[threadIdx.x];
  __syncthreads();
  const float half_n = 0.5f * (float)N;
  const int64_t nn = (int64_t)N * N;
  const float* Nr = Num + row * ld_pix;
  const float inv_d = (mode == EMC_COMPRESS_IDW) ? 1.0f / dj : 1.0f;
  const float dv = (mode == EMC_COMPRESS_IDW) ? 1.0f : dj;
  // every column with geometry: pixels (w = 1) and duplicate columns carrying
  // counts above 256 (w = kDupMark), which add numerator but no denominator
  for (int64_t i = threadIdx.x; i < ld_pix; i += kCompressThreads) {
    float4 a = qh[i], b = ql[i];
    if (a.w == 0.f) continue;
    int f[3];
    float t[3];
    rotate_to_grid(R, a, b, half_n, f, t);
    const float v = Nr[i] * inv_d;
    const float dvi = a.w == 1.f ? dv : 0.f;
    if constexpr (INTERIOR) {
      const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
      const int nn32 = N * N;
      const int base = f[0] * nn32 + f[1] * N + f[2];
#pragma unroll
      for (int c = 0; c < 8; c++) {
        const int cx = (c >> 2) & 1, cy = (c >> 1) & 1, cz = c & 1;
        const float w = wx[cx] * wy[cy] * wz[cz];
        if (w == 0.f) continue;
        const int l = base + cx * nn32 + cy * N + cz;
        atomicAdd(g_num + l, (double)(w * v));
        if (dvi != 0.f) atomicAdd(g_den + l, (double)(w * dvi));
      }
    } else {
#pragma unroll
      for (int c = 0; c < 8; c++) {
        int x = f[0] + ((c >> 2) & 1), y = f[1] + ((c >> 1) & 1), z = f[2] + (c & 1);
        if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= N) continue;
        float w = (((c >> 2) & 1) ? t[0] : 1.f - t[0]) * (((c >> 1) & 1) ? t[1] : 1.f - t[1]) *
                  ((c & 1) ? t[2] : 1.f - t[2]);
        if (w == 0.f) continue;
        int64_t l = (int64_t)x * nn + (int64_t)y * N + z;
        // FP32 products (relative error 6e-8), FP64 accumulation in L2
        atomicAdd(g_num + l, (double)(w * v));
        if (dvi != 0.f) atomicAdd(g_den + l, (double)(w * dvi));
      }
    }
  }
}

cudaError_t launch_compress(const Geom& g, const RotDF* rot, int64_t nrot, const float* Num,
                            const float* den, int mode, double* g_num, double* g_den, int nrep,
                            cudaStream_t s) {
  if (nrot <= 0) return cudaSuccess;
  const int64_t n_vox = (int64_t)g.N * g.N * g.N;
  if (g.interior)
    compress_kernel<true><<<(unsigned)nrot, kCompressThreads, 0, s>>>(
        g.qh, g.ql, g.n_pix, g.ld_pix, g.N, rot, Num, den, mode, g_num, g_den, nrep, n_vox);
  else
    compress_kernel<false><<<(unsigned)nrot, kCompressThreads, 0, s>>>(
        g.qh, g.ql, g.n_pix, g.ld_pix, g.N, rot, Num, den, mode, g_num, g_den, nrep, n_vox);
  return cudaGetLastError();
}

}  // namespace emc
