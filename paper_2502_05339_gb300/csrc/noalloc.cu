// dmd_predict_noalloc: frame prediction for callers that must not allocate
// GPU memory.
//
// An interactive application (a game or editor driving the fluid from its
// frame loop) often reserves its GPU memory once at start-up under its own
// allocator and forbids allocation afterwards: cudaMalloc / cudaFree can
// synchronise the whole device and stall a frame, and a host that embeds this
// library as a plug-in may give it no allocator at all.  Such a caller still
// owns its inputs (Phi_R, modal, k, u) and the output frames, but it cannot
// provide the temporary workspace dmd_predict needs (coefficient matrix,
// split coefficient chunks, control rollout).  This entry point takes that
// workspace from a fixed array in the library's own device memory instead.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds DMD_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Calls are limited to problems whose forward-prediction workspace fits in it.
#include <mutex>

#include "common.cuh"

namespace dmd {
dmd_status predict_forward_workspace_bytes(const dmd_predict_desc* desc, size_t* bytes);
dmd_status predict_forward(const dmd_predict_desc* desc, const float* Phi_R, const double* modal, const int32_t* k,
                           const float* u, float* out, void* workspace, size_t ws_bytes, cudaStream_t st,
                           const char* who);
}  // namespace dmd

namespace {

static __device__ __align__(256) unsigned char g_predict_scratch[DMD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_predict_scratch on the current device.  In host code
// the name g_predict_scratch is only a handle for the runtime, not a device
// address; cudaGetSymbolAddress translates it, once per device.
dmd_status scratch_address(void** out) {
  int dev = -1;
  DMD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    ::dmd::set_error("dmd_predict_noalloc: device ordinal %d out of range (max %d)", dev, kMaxDevices - 1);
    return DMD_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_predict_scratch);
    if (e != cudaSuccess || p == nullptr) {
      ::dmd::set_error("dmd_predict_noalloc: cudaGetSymbolAddress of the scratch array failed on device %d: %s", dev,
                       cudaGetErrorString(e));
      return DMD_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DMD_OK;
}

}  // namespace

extern "C" dmd_status dmd_predict_noalloc(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                                          const int32_t* k, const float* u, float* out, void* stream) {
  size_t need = 0;
  DMD_TRY(::dmd::predict_forward_workspace_bytes(desc, &need));
  if (need > (size_t)DMD_NOALLOC_SCRATCH_BYTES) {
    ::dmd::set_error(
        "dmd_predict_noalloc: this problem needs %zu bytes of workspace, more than the fixed %zu-byte scratch "
        "array; call dmd_predict with a caller-provided workspace instead",
        need, (size_t)DMD_NOALLOC_SCRATCH_BYTES);
    return DMD_EINVAL;
  }
  void* scratch = nullptr;
  DMD_TRY(scratch_address(&scratch));
  // The array keeps whatever the previous call left in it: start from zeros
  // so that no entry of this call's coefficients can come from that call.
  DMD_CUDA_TRY(cudaMemsetAsync(scratch, 0, need, (cudaStream_t)stream));
  return ::dmd::predict_forward(desc, Phi_R, modal, k, u, out, scratch, need, (cudaStream_t)stream,
                                "dmd_predict_noalloc");
}
