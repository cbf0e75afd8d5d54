// noalloc.cu -- emc_loglik_static: the E-step pass 1 for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a host
// application or framework that owns every device allocation and hands out
// only the buffers it created, in a process whose memory pool is already
// committed, or on a path that must not block on the allocator. Such a caller
// can pass its inputs and outputs but cannot provide the workspace that
// emc_ctx_create needs. This entry point keeps the only scratch the pass needs
// (the per-tile (max, sum) pairs the final merge reads) in a file-scope device
// array that is part of the library image, so nothing is allocated at call
// time: no cudaMalloc, no cudaFree, no allocating library routine.
//
// Costs and limits: every GPU that loads libemc holds kStaticScratchBytes of
// it until the process exits. The array is shared by all calls and keeps the
// last call's contents; calls that overlap on the GPU (different streams, or
// different host threads on one device) race on it and must be serialised by
// the caller. The first call on a device looks the array's device address up
// (cudaGetSymbolAddress) with that device current and keeps it for the life of
// the process; make that first call before any stream capture, and do not use
// the call after cudaDeviceReset (the kept address would be stale).
#include <mutex>

#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {
namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_loglik_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loglik_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

int64_t up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace
}  // namespace emc

using namespace emc;

extern "C" int emc_loglik_static(const emc_config* cfg, const void* L, const double* bias,
                                 const uint16_t* frames, int64_t nrot, double* lse_m,
                                 double* lse_s, int accumulate, int32_t* device_status,
                                 emc_stream stream) {
  if (!cfg || !L || !bias || !frames || !lse_m || !lse_s) return EMC_ERR_ARG;
  if (cfg->n_pix < 1 || cfg->n_data < 1 || nrot < 1 || nrot > cfg->n_rot) return EMC_ERR_ARG;
  if (cfg->n_pix > (1LL << 24) || cfg->n_rot > (1LL << 31) || cfg->n_data > (1LL << 31))
    return EMC_ERR_ARG;
  // the tensor maps need 16-byte aligned bases; the FP64 arrays, 8-byte ones
  if ((((uintptr_t)L) & 15) || (((uintptr_t)frames) & 15) || (((uintptr_t)bias) & 7) ||
      (((uintptr_t)lse_m) & 7) || (((uintptr_t)lse_s) & 7) || (((uintptr_t)device_status) & 3))
    return EMC_ERR_ARG;
  if (cfg->precision < EMC_PREC_FP32 || cfg->precision > EMC_PREC_FP16_SPLIT) return EMC_ERR_ARG;
  if (cfg->model != EMC_MODEL_POISSON || (cfg->flags & EMC_FLAG_WIDE_COUNTS))
    return EMC_ERR_UNSUPPORTED;
  const int64_t ld_pix = up(cfg->n_pix + 1, 64);
  const int64_t ld_data = up(cfg->n_data, 256);
  const int64_t rows = up(nrot, 128);
  // per 64-row tile one double and one float per frame; blocks of rows that fit
  const int64_t per_tile = ld_data * (int64_t)(sizeof(double) + sizeof(float));
  int64_t block = (int64_t)(kStaticScratchBytes / per_tile) * 64 / 128 * 128;
  if (block < 128) return EMC_ERR_UNSUPPORTED;  // frames beyond what the static scratch holds
  if (block > rows) block = rows;

  void* base = nullptr;
  if (scratch_ptr(&base) != cudaSuccess) return EMC_ERR_CUDA;
  double* part_m = reinterpret_cast<double*>(base);
  float* part_s = reinterpret_cast<float*>(part_m + (block / 64) * ld_data);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t elem = cfg->precision == EMC_PREC_FP32 ? 4 : 2;
  for (int64_t r0 = 0; r0 < rows; r0 += block) {
    const int64_t nb = block < rows - r0 ? block : rows - r0;
    const char* Lb = reinterpret_cast<const char*>(L) + (size_t)r0 * ld_pix * elem;
    int64_t tiles;
    cudaError_t e;
    if (cfg->precision == EMC_PREC_FP32) {
      e = launch_simt_pass1(reinterpret_cast<const float*>(Lb), ld_pix, bias + r0, nb, frames,
                            ld_data, cfg->n_data, part_m, part_s, nullptr, nullptr, s);
      tiles = simt_pass1_tiles(nb);
    } else {
      Planes p{const_cast<char*>(Lb), rows * ld_pix, ld_pix};
      e = launch_tc_pass1(p, cfg->precision, bias + r0, nb, frames, ld_data, cfg->n_data, ld_pix, part_m,
                          part_s, nullptr, nullptr, nullptr, nullptr, device_status, s);
      tiles = tc_pass1_tiles(nb);
    }
    if (e != cudaSuccess) return EMC_ERR_CUDA;
    e = launch_lse_merge(part_m, part_s, tiles, ld_data, cfg->n_data, lse_m, lse_s,
                         (accumulate || r0 > 0) ? 1 : 0, 0, device_status, s);
    if (e != cudaSuccess) return EMC_ERR_CUDA;
  }
  return EMC_OK;
}
