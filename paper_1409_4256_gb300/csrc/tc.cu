// tc.cu -- tcgen05 forms of the Maximize step (placeholder until the tensor-core kernels land).
#include "emc_common.cuh"
#include "emc_internal.h"

namespace emc {

int64_t tc_pass1_tiles(int64_t rows) { return rows / 128; }

cudaError_t launch_tc_pass1(const Planes&, int, const double*, int64_t, const uint16_t*, int64_t,
                            int64_t, int64_t, double*, float*, int32_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_tc_normalize(const Planes&, int, const double*, int64_t, int64_t,
                                const uint16_t*, int64_t, int64_t, int64_t, const double*,
                                const double*, Planes, int32_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_tc_update(const Planes&, int64_t, const uint16_t*, int64_t, int64_t, int64_t,
                             float*, float*, int32_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace emc
