// Householder reductions of the fit's small FP64 matrices spread over a
// thread-block cluster (sm_103a).
//
// GB300 runs FP64 at about 2 DFMA per clock per SM, so a one-CTA reduction of
// a 150 x 150 matrix is bound by a single SM's FP64 pipe (10/3 n^3 flops for
// the Hessenberg form).  Here the matrix is spread over the CL CTAs of one
// cluster, column j owned by CTA j % CL (cyclic, so the shrinking active part
// stays balanced), and every step exchanges only vectors through distributed
// shared memory:
//
//   Hessenberg (A <- Q^T A Q, Sec. 3.1's reduced operator before the Francis
//   QR), step k, reflector H_k = I - tau v v^T on indices k+1 .. n-1:
//     1. the owner of column k forms v and tau from A[k+1.., k] and writes
//        them into every CTA's shared memory;                 cluster barrier
//     2. each CTA applies H_k from the left to its columns (column-local),
//        then forms its part of y = A v over its columns and writes it into
//        every CTA's shared memory;                           cluster barrier
//     3. each CTA sums the parts (fixed order: the same y in every CTA) and
//        applies H_k from the right to its columns.
//   Tridiagonalisation of a symmetric matrix (the eigendecomposition of
//   B B^T, the SVD of Sec. 4.3's B), step k:
//     1. as above;                                            cluster barrier
//     2. each CTA forms p_j = tau A22[:, j] . v for its columns and writes
//        them into every CTA's shared memory;                 cluster barrier
//     3. each CTA forms w = p - (tau/2)(p . v) v (same order everywhere) and
//        applies A22 -= v w^T + w v^T to its columns.
// The vector buffers are double-buffered by step parity, so two cluster
// barriers per step suffice.  The reflector storage (v below the subdiagonal
// of column k, tau[k], beta on the subdiagonal) is that of the one-CTA
// kernels, so the Francis QR, the inverse iterations and the
// back-transformation read the result unchanged.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace dmd {

namespace {

constexpr int CL = 8;             // CTAs per cluster (portable size)
constexpr int CL_THREADS = 256;

// Householder scalars of x[0..m) (x[0] = alpha), as the one-CTA kernels take
// them: beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta, v = x / (alpha - beta)
// with v[0] = 1; tau = 0 when x[1..m) is zero.
__device__ __forceinline__ void house_scalars(double alpha, double sig, double& tau, double& beta, double& sc) {
  if (sig == 0.0) {
    tau = 0.0;
    beta = alpha;
    sc = 0.0;
  } else {
    const double nrm = sqrt(alpha * alpha + sig);
    beta = alpha <= 0.0 ? nrm : -nrm;
    tau = (beta - alpha) / beta;
    sc = 1.0 / (alpha - beta);
  }
}

// Owner's part of step k: reflector of its local column k, broadcast of v
// (vb[buf] of every CTA) and of (tau, beta) (sc[2 buf .. 2 buf + 1] of every
// CTA), reflector storage in the column and tau[k] in global memory.
__device__ __forceinline__ void owner_reflector(cg::cluster_group& cl, int n, int k, double* col, double* vbuf,
                                               double* scal, int buf, double* red, double* tau_out) {
  const int tid = threadIdx.x, bd = blockDim.x;
  const int m = n - k - 1;
  double* x = col + (k + 1);
  double loc = 0.0;
  for (int i = 1 + tid; i < m; i += bd) loc += x[i] * x[i];
  const double sig = block_sum(loc, red);
  double t, beta, sc;
  house_scalars(x[0], sig, t, beta, sc);
  for (int i = tid; i < m; i += bd) {
    const double vi = (i == 0) ? 1.0 : x[i] * sc;
    for (int r = 0; r < CL; ++r) cl.map_shared_rank(vbuf, r)[i] = vi;
  }
  if (tid == 0) {
    for (int r = 0; r < CL; ++r) {
      double* s = cl.map_shared_rank(scal, r);
      s[2 * buf] = t;
      s[2 * buf + 1] = beta;
    }
    tau_out[k] = t;
  }
  __syncthreads();   // every thread has read x before it is overwritten
  if (t != 0.0) {
    for (int i = 1 + tid; i < m; i += bd) x[i] = x[i] * sc;
    if (tid == 0) x[0] = beta;
  }
}

__device__ __forceinline__ void load_cols(double* S, int ldw, const double* A, int ld, int n, int c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int jl = warp; c + CL * jl < n; jl += nw)
    for (int i = lane; i < n; i += 32) S[i + jl * ldw] = A[i + (int64_t)(c + CL * jl) * ld];
}
__device__ __forceinline__ void store_cols(double* A, int ld, const double* S, int ldw, int n, int c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int jl = warp; c + CL * jl < n; jl += nw)
    for (int i = lane; i < n; i += 32) A[i + (int64_t)(c + CL * jl) * ld] = S[i + jl * ldw];
}

// First local column index whose global column is >= j0.
__device__ __forceinline__ int first_local(int j0, int c) { return j0 <= c ? 0 : (j0 - c + CL - 1) / CL; }

// Shared memory: S (n x ceil(n / CL), ld n | 1), vb[2][n], yp[2][CL][n], red[32], scal[4].
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CL_THREADS)
    k_hessenberg_cl(int n, double* A, int ld, double* tau) {
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int ldw = n | 1, ncl = (n + CL - 1) / CL;
  extern __shared__ double sm[];
  double* S = sm;
  double* vb = S + (size_t)ldw * ncl;
  double* yp = vb + 2 * n;
  double* red = yp + 2 * CL * n;
  double* scal = red + 32;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  load_cols(S, ldw, A, ld, n, c);
  __syncthreads();
  cl.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1, buf = k & 1;
    double* v = vb + buf * n;
    if (k % CL == c) owner_reflector(cl, n, k, S + (k / CL) * ldw, v, scal, buf, red, tau);
    cl.sync();
    const double t = scal[2 * buf];
    const int j0 = first_local(k + 1, c);
    if (t != 0.0) {
      // left: A[k+1.., j] -= t v (v . A[k+1.., j]), one warp per local column
      for (int jl = j0 + warp; jl < ncl && c + CL * jl < n; jl += nw) {
        double* col = S + jl * ldw + (k + 1);
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s = fma(col[i], v[i], s);
        const double tw = t * warp_sum(s);
        for (int i = lane; i < m; i += 32) col[i] = fma(-v[i], tw, col[i]);
      }
      __syncthreads();
      // this CTA's part of y = A[:, k+1..] v, to every CTA
      for (int i = tid; i < n; i += bd) {
        double s = 0.0;
        for (int jl = j0; jl < ncl && c + CL * jl < n; ++jl) s = fma(S[i + jl * ldw], v[c + CL * jl - k - 1], s);
        for (int r = 0; r < CL; ++r) cl.map_shared_rank(yp, r)[(buf * CL + c) * n + i] = s;
      }
    }
    cl.sync();
    if (t != 0.0) {
      // right: A[:, j] -= t y v_j for the local columns j > k
      for (int i = tid; i < n; i += bd) {
        double y = 0.0;
        for (int r = 0; r < CL; ++r) y += yp[(buf * CL + r) * n + i];
        const double ty = t * y;
        for (int jl = j0; jl < ncl && c + CL * jl < n; ++jl)
          S[i + jl * ldw] = fma(-ty, v[c + CL * jl - k - 1], S[i + jl * ldw]);
      }
    }
    __syncthreads();
  }
  if (c == 0 && tid == 0) {
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) tau[k] = 0.0;
  }
  store_cols(A, ld, S, ldw, n, c);
  cl.sync();   // no CTA leaves while another may still write into its shared memory
}

// Symmetric A (both triangles) -> tridiagonal, same storage as k_sytrd.
// Shared memory: S (n x ceil(n / CL)), vb[2][n], pf[2][n], red[32], scal[4].
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CL_THREADS)
    k_sytrd_cl(int n, double* A, int ld, double* tau) {
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int ldw = n | 1, ncl = (n + CL - 1) / CL;
  extern __shared__ double sm[];
  double* S = sm;
  double* vb = S + (size_t)ldw * ncl;
  double* pf = vb + 2 * n;
  double* red = pf + 2 * n;
  double* scal = red + 32;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  load_cols(S, ldw, A, ld, n, c);
  __syncthreads();
  cl.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1, buf = k & 1;
    double* v = vb + buf * n;
    double* p = pf + buf * n;
    if (k % CL == c) owner_reflector(cl, n, k, S + (k / CL) * ldw, v, scal, buf, red, tau);
    cl.sync();
    const double t = scal[2 * buf];
    const int j0 = first_local(k + 1, c);
    if (t != 0.0) {
      // the symmetric partner of the subdiagonal: A[k, k+1] = beta
      if ((k + 1) % CL == c && tid == 0) S[k + ((k + 1) / CL) * ldw] = scal[2 * buf + 1];
      // p_j = t A22[:, j] . v for the local columns j > k, to every CTA
      for (int jl = j0 + warp; jl < ncl && c + CL * jl < n; jl += nw) {
        const double* col = S + jl * ldw + (k + 1);
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s = fma(col[i], v[i], s);
        s = t * warp_sum(s);
        if (lane < CL) cl.map_shared_rank(pf, lane)[buf * n + (c + CL * jl - k - 1)] = s;
      }
    }
    cl.sync();
    if (t != 0.0) {
      // w = p - (t / 2)(p . v) v, the same in every CTA
      double loc = 0.0;
      for (int i = tid; i < m; i += bd) loc = fma(p[i], v[i], loc);
      const double pv = block_sum(loc, red);
      const double h = 0.5 * t * pv;
      // A22[:, j] -= v w_j + w v_j for the local columns (w formed on the fly)
      for (int jl = j0 + warp; jl < ncl && c + CL * jl < n; jl += nw) {
        const int jj = c + CL * jl - k - 1;
        const double wj = fma(-h, v[jj], p[jj]), vj = v[jj];
        double* col = S + jl * ldw + (k + 1);
        for (int i = lane; i < m; i += 32) {
          const double wi = fma(-h, v[i], p[i]);
          col[i] -= fma(v[i], wj, wi * vj);
        }
      }
    }
    __syncthreads();
  }
  if (c == 0 && tid == 0) {
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) tau[k] = 0.0;
  }
  store_cols(A, ld, S, ldw, n, c);
  cl.sync();
}

}  // namespace

// Cluster versions are used from this size up (smaller matrices stay on one CTA).
bool householder_cluster_fits(int n) { return n >= 32 && n <= 256; }

dmd_status hessenberg_cluster(int n, double* A, int ld, double* tau, cudaStream_t st) {
  const int ncl = (n + CL - 1) / CL;
  const size_t smem = ((size_t)(n | 1) * ncl + 2 * (size_t)n + 2 * (size_t)CL * n + 36) * sizeof(double);
  if (smem > 48 * 1024)
    DMD_CUDA_TRY(cudaFuncSetAttribute(k_hessenberg_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_hessenberg_cl<<<CL, CL_THREADS, smem, st>>>(n, A, ld, tau);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status sytrd_cluster(int n, double* A, int ld, double* tau, cudaStream_t st) {
  const int ncl = (n + CL - 1) / CL;
  const size_t smem = ((size_t)(n | 1) * ncl + 4 * (size_t)n + 36) * sizeof(double);
  if (smem > 48 * 1024)
    DMD_CUDA_TRY(cudaFuncSetAttribute(k_sytrd_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sytrd_cl<<<CL, CL_THREADS, smem, st>>>(n, A, ld, tau);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

}  // namespace dmd
