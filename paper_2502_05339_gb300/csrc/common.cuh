// Shared host/device helpers of libdmd (no method arithmetic lives here).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/dmd.h"

namespace dmd {

// ---------------------------------------------------------------- host errors

void set_error(const char* fmt, ...);

#define DMD_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::dmd::set_error("%s:%d: %s -> %s", __FILE__, __LINE__, #expr,               \
                       cudaGetErrorString(_e));                                    \
      return DMD_ECUDA;                                                            \
    }                                                                              \
  } while (0)

void count_launch();

#define DMD_LAUNCH_CHECK()                                                         \
  do {                                                                             \
    ::dmd::count_launch();                                                         \
    cudaError_t _e = cudaGetLastError();                                           \
    if (_e != cudaSuccess) {                                                       \
      ::dmd::set_error("%s:%d: launch failed: %s", __FILE__, __LINE__,             \
                       cudaGetErrorString(_e));                                    \
      return DMD_ECUDA;                                                            \
    }                                                                              \
  } while (0)

#define DMD_TRY(expr)                                                              \
  do {                                                                             \
    dmd_status _s = (expr);                                                        \
    if (_s != DMD_OK) return _s;                                                   \
  } while (0)

#define DMD_REQUIRE(cond, ...)                                                     \
  do {                                                                             \
    if (!(cond)) {                                                                 \
      ::dmd::set_error(__VA_ARGS__);                                               \
      return DMD_EINVAL;                                                           \
    }                                                                              \
  } while (0)

// Status word that the bounded device waits report to (DMD_ETIMEOUT): for
// kernels launched from this host thread while a StatusScope is open, the
// running entry point's info (the fits); otherwise the current device's
// asynchronous status word, which dmd_async_status reads and clears.
int32_t* status_word();
int32_t* async_status_word();

class StatusScope {
 public:
  explicit StatusScope(int32_t* word);
  ~StatusScope();
  StatusScope(const StatusScope&) = delete;
  StatusScope& operator=(const StatusScope&) = delete;

 private:
  int32_t* prev_;
};

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t ceil_div(int64_t x, int64_t a) { return (x + a - 1) / a; }

// Bump allocator over a caller-provided workspace.  In "measure" mode (base ==
// nullptr) it only accumulates the size, so the size query and the real carve
// run the same code and can never disagree.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  template <class T>
  T* take(size_t count, size_t align = 256) {
    used = (size_t)round_up((int64_t)used, (int64_t)align);
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += count * sizeof(T);
    return p;
  }
  bool overflow() const { return base != nullptr && used > cap; }
};

// ------------------------------------------------------------- device helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; `red` must hold blockDim.x / 32 doubles.  All threads get the result.
// The cross-warp step is a butterfly over the warps' partials (fixed order,
// so reproducible) rather than a running sum: FP64 adds have ~64 cycles of
// latency on GB300, and a chain of 16-32 of them would dominate.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  return warp_sum(lane < nw ? red[lane] : 0.0);
}

__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = red[0];
  for (int i = 1; i < nw; ++i) t = fmax(t, red[i]);
  return t;
}

// Record the first failure in the device status word (info[0]) and the
// failing index in info[4]; later failures do not overwrite the first.
__device__ __forceinline__ void raise_status(int32_t* info, int32_t code, int32_t where) {
  if (info == nullptr) return;
  if (atomicCAS(&info[0], (int32_t)DMD_OK, code) == DMD_OK) info[4] = where;
}

}  // namespace dmd
