// BF16x3 tcgen05 passes (placeholder until the tensor-core kernels land).
#include "common.cuh"

namespace dmd {

size_t umma_nn_workspace_bytes(int64_t, int, int) { return 256; }
size_t umma_tn_workspace_bytes(int64_t, int, int) { return 256; }

dmd_status umma_gemm_nn(int64_t, int, int, const float*, int64_t, const double*, float*, int64_t, void*,
                        cudaStream_t) {
  set_error("mixed BF16x3 precision is not available in this build");
  return DMD_EINVAL;
}

dmd_status umma_gemm_tn(int64_t, int, int, const float*, int64_t, const float*, int64_t, double*, void*,
                        cudaStream_t) {
  set_error("mixed BF16x3 precision is not available in this build");
  return DMD_EINVAL;
}

}  // namespace dmd
