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
bool householder_cluster_fits(int n) { return n >= 96 && n <= 256; }

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

// ----------------------------------------------------------------- Cholesky
//
// G (n x n, ld; upper triangle read) -> upper R with R^T R = G, strict lower
// part zeroed; the pivot rule of the one-CTA kernels: a pivot not above
// tau * max_i G_ii drops its direction (row j of R is zero, counted in
// info[5]); a non-finite pivot is DMD_ENONFINITE and an all-zero diagonal
// DMD_ENUMERIC (the factorisation then stops and leaves G as it is).
// Column b is owned by CTA b % CL.  Step j of the right-looking
// factorisation needs row j of the current matrix and pivot j; both are
// broadcast at the end of step j - 1 (each CTA sends its updated entries of
// row j, the owner of column j its pivot decision), so every step has one
// cluster barrier.  Real = double, or float for the near-identity Grams of
// the second CholeskyQR pass (input and output stay FP64).
namespace {

template <class Real>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CL_THREADS)
    k_cholesky_cl(int n, double* G, int ld, double tau, int32_t* info, int tag, const int32_t* __restrict__ skip) {
  // a device-side flag (iterative callers stop without a host round trip):
  // every CTA of the cluster reads the same value, before any barrier
  if (skip != nullptr && *skip != 0) return;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int ldw = n | 1, ncl = (n + CL - 1) / CL;
  extern __shared__ __align__(16) unsigned char smc[];
  Real* S = reinterpret_cast<Real*>(smc);                 // n x ncl (rows 0..b of local column b)
  Real* rowb = S + (size_t)ldw * ncl;                     // [2][n] row j of the current matrix
  const size_t pb_off = ((((size_t)ldw * ncl + 2 * (size_t)n) * sizeof(Real)) + 15) & ~(size_t)15;
  double* pb = reinterpret_cast<double*>(smc + pb_off);   // [2][4]: piv, ipiv, state
  double* dm = pb + 8;                                    // [CL] per-CTA max of the diagonal
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  // load the upper triangle of the local columns; this CTA's largest diagonal entry
  for (int jl = warp; c + CL * jl < n; jl += nw) {
    const int b = c + CL * jl;
    for (int a = lane; a <= b; a += 32) S[a + jl * ldw] = (Real)G[a + (int64_t)b * ld];
  }
  __shared__ double red[32];
  double loc = 0.0;
  for (int jl = tid; c + CL * jl < n; jl += bd) {
    const double d = G[(c + CL * jl) + (int64_t)(c + CL * jl) * ld];
    loc = (isfinite(loc) && isfinite(d)) ? fmax(loc, d) : (double)NAN;
  }
  // fmax drops NaN: carry non-finite diagonals explicitly
  {
    double v = loc;
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = (isfinite(v) && isfinite(u)) ? fmax(v, u) : (double)NAN;
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double t = red[0];
      for (int i = 1; i < nw; ++i) t = (isfinite(t) && isfinite(red[i])) ? fmax(t, red[i]) : (double)NAN;
      for (int r = 0; r < CL; ++r) cl.map_shared_rank(dm, r)[c] = t;
    }
  }
  __syncthreads();
  cl.sync();
  double dmax = dm[0];
  for (int r = 1; r < CL; ++r) dmax = (isfinite(dmax) && isfinite(dm[r])) ? fmax(dmax, dm[r]) : (double)NAN;
  const double floor_ = tau * dmax;

  // pivot decision of column j (by its owner, single thread): state 0 take,
  // 1 drop, 2 stop.  Broadcast with row j's entries of the owner.
  auto decide = [&](int j, int buf) {
    const double d = (double)S[j + (j / CL) * ldw];
    double piv = 0.0, ipiv = 0.0, state = 0.0;
    if (!isfinite(d) || !isfinite(dmax)) {
      raise_status(info, DMD_ENONFINITE, tag * 1000 + j);
      state = 2.0;
    } else if (!(dmax > 0.0)) {
      raise_status(info, DMD_ENUMERIC, tag * 1000 + j);
      state = 2.0;
    } else if (!(d > floor_)) {
      state = 1.0;
      if (info) atomicAdd(&info[5], 1);
    } else {
      ipiv = rsqrt(d);
      piv = d * ipiv;
    }
    for (int r = 0; r < CL; ++r) {
      double* p = cl.map_shared_rank(pb, r) + 4 * buf;
      p[0] = piv;
      p[1] = ipiv;
      p[2] = state;
    }
  };
  // broadcast this CTA's entries of row j (columns b >= j)
  auto send_row = [&](int j, int buf) {
    for (int jl = first_local(j, c) + tid; jl < ncl && c + CL * jl < n; jl += bd) {
      const Real v = S[j + jl * ldw];
      for (int r = 0; r < CL; ++r) cl.map_shared_rank(rowb, r)[buf * n + c + CL * jl] = v;
    }
  };
  if (n > 0) {
    send_row(0, 0);
    if (c == 0 && tid == 0) decide(0, 0);
  }
  cl.sync();
  bool stopped = false;
  for (int j = 0; j < n; ++j) {
    const int buf = j & 1;
    const double* p = pb + 4 * buf;
    if (p[2] == 2.0) {
      stopped = true;
      break;
    }
    const bool take = p[2] == 0.0;
    const Real ip = (Real)p[1];
    const Real* row = rowb + buf * n;
    const int j0 = first_local(j + 1, c);
    // R's row j in the local columns, and the owner's diagonal entry
    if (c == j % CL && tid == 0) S[j + (j / CL) * ldw] = (Real)p[0];
    for (int jl = j0 + tid; jl < ncl && c + CL * jl < n; jl += bd)
      S[j + jl * ldw] = take ? row[c + CL * jl] * ip : Real(0);
    // trailing update S[a, b] -= r_a r_b, j < a <= b, for the local columns b
    if (take) {
      for (int jl = j0 + warp; jl < ncl && c + CL * jl < n; jl += nw) {
        const int b = c + CL * jl;
        const Real rb = row[b] * ip;
        Real* col = S + jl * ldw;
        for (int a = j + 1 + lane; a <= b; a += 32) col[a] -= (row[a] * ip) * rb;
      }
    }
    __syncthreads();
    if (j + 1 < n) {
      send_row(j + 1, buf ^ 1);
      if (c == (j + 1) % CL && tid == 0) decide(j + 1, buf ^ 1);
    }
    cl.sync();
  }
  if (!stopped) {
    for (int jl = warp; c + CL * jl < n; jl += nw) {
      const int b = c + CL * jl;
      for (int a = lane; a < n; a += 32) G[a + (int64_t)b * ld] = a <= b ? (double)S[a + jl * ldw] : 0.0;
    }
  }
  cl.sync();
}

template <class Real>
dmd_status cholesky_cluster_t(int n, double* G, int ld, double tau, int32_t* info, int tag, const int32_t* skip,
                              cudaStream_t st) {
  const int ncl = (n + CL - 1) / CL;
  const size_t pb_off = ((((size_t)(n | 1) * ncl + 2 * (size_t)n) * sizeof(Real)) + 15) & ~(size_t)15;
  const size_t smem = pb_off + (8 + CL) * sizeof(double);
  if (smem > 48 * 1024)
    DMD_CUDA_TRY(cudaFuncSetAttribute(k_cholesky_cl<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_cholesky_cl<Real><<<CL, CL_THREADS, smem, st>>>(n, G, ld, tau, info, tag, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

}  // namespace

bool cholesky_cluster_fits(int n) { return n >= 96 && n <= 512; }

dmd_status cholesky_cluster(int n, double* G, int ld, double tau, int32_t* info, int tag, bool fp32,
                            const int32_t* skip, cudaStream_t st) {
  return fp32 ? cholesky_cluster_t<float>(n, G, ld, tau, info, tag, skip, st)
              : cholesky_cluster_t<double>(n, G, ld, tau, info, tag, skip, st);
}

}  // namespace dmd
