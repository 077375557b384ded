// Small element-wise steps between the stages of the fit.
#include <atomic>

#include "common.cuh"

namespace dmd {

namespace {

// Asynchronous status words of the entry points without an info argument
// (one copy per device, zero-initialised when the module loads).
__device__ int32_t g_async_status[DMD_INFO_WORDS];

thread_local int32_t* t_status = nullptr;

// sigma_i = sqrt(max(ev_i, 0)) for the r leading eigenvalues of B B^T
// (descending), inv_sq_i = 1 / ev_i; rank guard sigma_{r-1} > 1e-6 sigma_0.
__global__ void k_sigma(int l, int r, const double* ev, double* sigma, double* inv_sq, int32_t* info) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double s0 = sqrt(fmax(ev[0], 0.0));
  for (int i = 0; i < r; ++i) {
    const double e = fmax(ev[i], 0.0);
    const double s = sqrt(e);
    sigma[i] = s;
    if (!(s > 1e-6 * s0) || !isfinite(s)) {
      raise_status(info, isfinite(s) ? DMD_ERANK : DMD_ENONFINITE, 7000 + i);
      inv_sq[i] = 0.0;
    } else {
      inv_sq[i] = 1.0 / e;
    }
  }
  (void)l;
}

// Fallback gate of the CholeskyQR orthonormalisation.  mode 0: remember the
// dropped-direction count info[5]; mode 1: gate[1] = 1 (skip the fallback)
// unless more than `spare` directions were dropped since -- the sketch has
// spare = l - r columns beyond the requested rank, and directions dropped
// among those leave a basis of rank >= r -- else 0, and the count is
// restored, since the shifted fallback keeps every direction.
__global__ void k_gate(int32_t* info, int32_t* gate, int mode, int spare) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (mode == 0) {
    gate[0] = info[5];
    gate[1] = 1;
  } else {
    const bool short_of_rank = info[5] - gate[0] > spare;
    gate[1] = short_of_rank ? 0 : 1;
    if (short_of_rank) info[5] = gate[0];
  }
}

// G (n x n, ld) += s I with s = rel * max_i G_ii (skipped when *skip != 0).
__global__ void k_shift_diag(int n, double* G, int ld, double rel, const int32_t* skip) {
  if (*skip != 0) return;
  __shared__ double red[32];
  double loc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) loc = fmax(loc, G[i + (int64_t)i * ld]);
  const double s = rel * block_max(loc, red);
  for (int i = threadIdx.x; i < n; i += blockDim.x) G[i + (int64_t)i * ld] += s;
}

__global__ void k_scale_cols(int rows, int cols, double* A, int lda, const double* s) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * cols) return;
  const int i = (int)(t % rows), j = (int)(t / rows);
  A[(int64_t)j * lda + i] *= s[j];
}

__global__ void k_check_finite(int64_t count, const double* A, int32_t* info, int tag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count && !isfinite(A[t])) raise_status(info, DMD_ENONFINITE, tag);
}

__global__ void k_maxabs(int64_t count, const double* A, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) v = fmax(v, fabs(A[t]));
  v = block_max(v, red);
  if (threadIdx.x == 0) *out = v;
}

__global__ void k_copy(int64_t count, const double* src, double* dst) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count) dst[t] = src[t];
}

// Om[:, j] = [P[0:l, j]; Ups[:, j]] (column-major, ld l + q)
__global__ void k_stack(int l, int q, int m, const double* P, const float* Ups, double* Om) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int L = l + q;
  if (t >= (int64_t)L * m) return;
  const int i = (int)(t % L), j = (int)(t / L);
  Om[t] = (i < l) ? P[(int64_t)j * l + i] : (double)Ups[(int64_t)j * q + (i - l)];
}

// inv_sq[i] = 1 / ev[i] for the p leading eigenvalues (descending) of a Gram
// matrix; rank guard sqrt(ev[p-1]) > 1e-6 sqrt(ev[0]); optional sigma output.
__global__ void k_sigma_range(int L, int p, const double* ev, double* sigma, double* inv_sq, int32_t* info, int tag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double s0 = sqrt(fmax(ev[0], 0.0));
  for (int i = 0; i < p; ++i) {
    const double e = fmax(ev[i], 0.0);
    const double s = sqrt(e);
    if (sigma) sigma[i] = s;
    if (!(s > 1e-6 * s0) || !isfinite(s)) {
      raise_status(info, isfinite(s) ? DMD_ERANK : DMD_ENONFINITE, tag + i);
      inv_sq[i] = 0.0;
    } else {
      inv_sq[i] = 1.0 / e;
    }
  }
  (void)L;
}

__global__ void k_fill_int(int64_t count, int* dst, int v) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count) dst[t] = v;
}

}  // namespace

dmd_status fit_glue_sigma(int l, int r, const double* ev, double* sigma, double* inv_sq, int32_t* info,
                          cudaStream_t st) {
  k_sigma<<<1, 32, 0, st>>>(l, r, ev, sigma, inv_sq, info);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_scale_cols(int rows, int cols, double* A, int lda, const double* s, cudaStream_t st) {
  const int64_t tot = (int64_t)rows * cols;
  if (tot == 0) return DMD_OK;
  k_scale_cols<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(rows, cols, A, lda, s);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_check_finite(int64_t count, const double* A, int32_t* info, int tag, cudaStream_t st) {
  if (count == 0) return DMD_OK;
  k_check_finite<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, A, info, tag);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_maxabs(int64_t count, const double* A, double* out, cudaStream_t st) {
  k_maxabs<<<1, 256, 0, st>>>(count, A, out);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_copy(int64_t count, const double* src, double* dst, cudaStream_t st) {
  if (count == 0) return DMD_OK;
  k_copy<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, src, dst);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_stack(int l, int q, int m, const double* P, const float* Ups, double* Om, cudaStream_t st) {
  const int64_t tot = (int64_t)(l + q) * m;
  k_stack<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(l, q, m, P, Ups, Om);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_sigma_range(int L, int p, const double* ev, double* sigma, double* inv_sq, int32_t* info, int tag,
                                cudaStream_t st) {
  k_sigma_range<<<1, 32, 0, st>>>(L, p, ev, sigma, inv_sq, info, tag);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_gate(int32_t* info, int32_t* gate, int mode, int spare, cudaStream_t st) {
  k_gate<<<1, 32, 0, st>>>(info, gate, mode, spare);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_shift_diag(int n, double* G, int ld, double rel, const int32_t* skip, cudaStream_t st) {
  k_shift_diag<<<1, 256, 0, st>>>(n, G, ld, rel, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status fit_glue_fill_int(int64_t count, int* dst, int v, cudaStream_t st) {
  if (count == 0) return DMD_OK;
  k_fill_int<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, dst, v);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

int32_t* async_status_word() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int32_t*> addr[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  int32_t* a = addr[dev].load(std::memory_order_acquire);
  if (a == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_async_status) != cudaSuccess) return nullptr;
    a = static_cast<int32_t*>(p);
    addr[dev].store(a, std::memory_order_release);
  }
  return a;
}

int32_t* status_word() { return t_status != nullptr ? t_status : async_status_word(); }

StatusScope::StatusScope(int32_t* word) : prev_(t_status) { t_status = word; }
StatusScope::~StatusScope() { t_status = prev_; }

}  // namespace dmd
