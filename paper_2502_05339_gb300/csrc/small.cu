// FP64 small dense linear algebra on the device (sizes l, r <= a few hundred).
//
// These are the l x l / r x r steps of the fit: the Cholesky factors of
// CholeskyQR2 (Sec. 4.3 range finder), the SVD of B = Q^T X (Sec. 4.3) taken
// through the eigendecomposition of B B^T, the eigendecomposition of the
// reduced operator A~ (Sec. 3.1), and the least-squares amplitudes
// b = Phi^+ x_0 (Eq. projection).  Algorithms (all textbook, written here from
// their mathematical statement):
//   * Cholesky: right-looking, upper factor R with R^T R = G.
//   * Hessenberg reduction by Householder reflectors (a symmetric input gives
//     a tridiagonal matrix).
//   * Eigenvalues of an upper Hessenberg matrix: Francis implicit double-shift
//     QR with 3x3 reflectors, deflation on negligible subdiagonals and
//     exceptional shifts (Golub & Van Loan, Sec. 7.5).
//   * Eigenvectors: inverse iteration with the computed eigenvalue as shift on
//     the Hessenberg (complex shift) or tridiagonal (real shift) matrix, then
//     back-transformation with the Hessenberg reflectors.
//   * Symmetric tridiagonal eigenvalues: bisection on Sturm counts.
//   * Least squares: Householder QR and back substitution.
// Every kernel that can fail writes DMD_ENUMERIC / DMD_ENONFINITE to info[0].
#include <float.h>

#include <type_traits>

#include "common.cuh"

namespace dmd {

namespace {

constexpr double kEps = DBL_EPSILON;

// ------------------------------------------------------ FP64 reciprocal

// 1 / x for finite, nonzero, normal x: the hardware's approximate reciprocal
// (about 20 correct bits) refined by two Newton-Raphson steps
// y <- y + y (1 - x y), each of which roughly doubles the correct bits.  An
// IEEE FP64 division is a long dependent sequence on GB300 (measured ~560
// cycles); this is one approximation and four FMAs.  Used inside sequential
// recurrences (Sturm counts, the Hessenberg LU of the eigenvector
// refinement), where that latency is the critical path.
__device__ __forceinline__ double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// 1 / sqrt(x) for finite x > 0 (normal): the hardware's approximate
// reciprocal square root refined by two Newton-Raphson steps
// y <- y (3/2 - x/2 y^2) (quadratic convergence: ~22 -> ~44 -> full bits).
// Replaces a square root followed by a division (~1250 cycles of dependent
// FP64 latency on GB300) on the Cholesky's sequential pivot path.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = 0.5 * x;
  y = y * fma(-h, y * y, 1.5);
  return y * fma(-h, y * y, 1.5);
}

// ------------------------------------------------------------------ GEMM

// C[M x N] = alpha op(A) op(B) + beta C (column-major; op = transpose when t* != 0).
// Kernels that take `skip` return at once when it is non-NULL and *skip != 0
// (a device-side flag: iterative solvers stop without a host round trip).
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A,
                                               int lda, int ta, const double* __restrict__ B, int ldb,
                                               int tb, double beta, double* __restrict__ C, int ldc,
                                               const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    {
      const int i = i0 + tx, k = k0 + ty;
      double v = 0.0;
      if (i < M && k < K) v = ta ? A[(int64_t)i * lda + k] : A[(int64_t)k * lda + i];
      As[ty][tx] = v;
    }
    {
      const int k = k0 + tx, j = j0 + ty;
      double v = 0.0;
      if (k < K && j < N) v = tb ? B[(int64_t)k * ldb + j] : B[(int64_t)j * ldb + k];
      Bs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[kk][tx], Bs[ty][kk], acc);
    __syncthreads();
  }
  const int i = i0 + tx, j = j0 + ty;
  if (i < M && j < N) {
    double* c = C + (int64_t)j * ldc + i;
    *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * (*c);
  }
}

// ------------------------------------------------------------- Cholesky

// In place: the upper triangle of G (n x n, ld) becomes R with R^T R = G; the
// strict lower triangle is zeroed.  One CTA.  Column j whose pivot (the
// squared residual of column j against columns 0..j-1) is not above
// tau * max_i G_ii is dropped: row j of R is set to zero, so the Gram-based
// orthonormalisation leaves that (numerically dependent) direction out;
// k_tri_inv_upper then zeroes row and column j of R^{-1}.  Drops are counted
// in info[5].  A non-finite pivot is DMD_ENONFINITE, an all-zero matrix
// DMD_ENUMERIC.
__global__ void k_cholesky_upper(int n, double* G, int ld, double tau, int32_t* info, int tag,
                                 const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ double piv;
  __shared__ double red[32];
  const int tid = threadIdx.x, bd = blockDim.x;
  double loc = 0.0;
  for (int j = tid; j < n; j += bd) loc = fmax(loc, G[j + (int64_t)j * ld]);
  const double dmax = block_max(loc, red);
  const double floor_ = tau * dmax;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = G[j + (int64_t)j * ld];
      if (!isfinite(d) || !isfinite(dmax)) {
        raise_status(info, DMD_ENONFINITE, tag * 1000 + j);
        piv = -1.0;
      } else if (!(dmax > 0.0)) {
        raise_status(info, DMD_ENUMERIC, tag * 1000 + j);
        piv = -1.0;
      } else if (!(d > floor_)) {
        piv = 0.0;   // dropped direction
        if (info) atomicAdd(&info[5], 1);
      } else {
        piv = sqrt(d);
      }
      if (piv >= 0.0) G[j + (int64_t)j * ld] = piv;
    }
    __syncthreads();
    const double p = piv;
    if (p < 0.0) return;
    if (p == 0.0) {
      for (int i = j + 1 + tid; i < n; i += bd) G[j + (int64_t)i * ld] = 0.0;
      __syncthreads();
      continue;
    }
    const double ip = 1.0 / p;
    for (int i = j + 1 + tid; i < n; i += bd) G[j + (int64_t)i * ld] *= ip;
    __syncthreads();
    const int w = n - j - 1;
    for (int e = tid; e < w * w; e += bd) {
      const int a = j + 1 + e % w, b = j + 1 + e / w;
      if (a <= b) G[a + (int64_t)b * ld] -= G[j + (int64_t)a * ld] * G[j + (int64_t)b * ld];
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += bd) {
    const int a = e % n, b = e / n;
    if (a > b) G[a + (int64_t)b * ld] = 0.0;
  }
}

// T = R^{-1} for upper triangular R by back substitution, one warp per
// column (the dot products are split across the lanes).  A zero diagonal
// entry marks a dropped direction: its row and column of T are zero.
__global__ void k_tri_inv_upper(int n, const double* __restrict__ R, int ldr, double* __restrict__ T, int ldt,
                                const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  double* t = T + (int64_t)j * ldt;
  for (int i = j + 1 + lane; i < n; i += 32) t[i] = 0.0;
  const double rjj = R[j + (int64_t)j * ldr];
  if (rjj == 0.0) {
    for (int i = lane; i <= j; i += 32) t[i] = 0.0;
    return;
  }
  if (lane == 0) t[j] = 1.0 / rjj;
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + lane; k <= j; k += 32) s = fma(R[i + (int64_t)k * ldr], t[k], s);
    s = warp_sum(s);
    if (lane == 0) {
      const double rii = R[i + (int64_t)i * ldr];
      t[i] = (rii == 0.0) ? 0.0 : -s / rii;
    }
    __syncwarp();
  }
}

// ------------------------------------------------- Hessenberg reduction

// A (n x n, ld) <- Q^T A Q upper Hessenberg, Q = H_0 ... H_{n-3},
// H_k = I - tau_k v v^T with v = [1, A[k+2.., k]] on indices k+1..n-1.
// Shared memory: 2n + 32 doubles.  One CTA.
__global__ void k_hessenberg(int n, double* A, int ld, double* tau) {
  extern __shared__ double sm[];
  double* v = sm;
  double* w = sm + n;
  double* red = sm + 2 * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = A + (int64_t)k * ld + (k + 1);
    double loc = 0.0;
    for (int i = 1 + tid; i < m; i += bd) loc += x[i] * x[i];
    const double sig = block_sum(loc, red);
    const double alpha = x[0];
    if (sig == 0.0) {
      if (tid == 0) tau[k] = 0.0;
      __syncthreads();
      continue;
    }
    const double nrm = sqrt(alpha * alpha + sig);
    const double beta = alpha <= 0.0 ? nrm : -nrm;
    const double t = (beta - alpha) / beta;
    const double sc = 1.0 / (alpha - beta);
    for (int i = tid; i < m; i += bd) v[i] = (i == 0) ? 1.0 : x[i] * sc;
    __syncthreads();
    for (int i = 1 + tid; i < m; i += bd) x[i] = v[i];
    if (tid == 0) {
      x[0] = beta;
      tau[k] = t;
    }
    // left: rows k+1.., columns k+1..
    for (int j = k + 1 + tid; j < n; j += bd) {
      const double* col = A + (int64_t)j * ld + (k + 1);
      double s = 0.0;
      for (int i = 0; i < m; ++i) s = fma(v[i], col[i], s);
      w[j] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += bd) {
      const int i = e % m, j = k + 1 + e / m;
      A[(int64_t)j * ld + (k + 1 + i)] -= t * v[i] * w[j];
    }
    __syncthreads();
    // right: all rows, columns k+1..
    for (int i = tid; i < n; i += bd) {
      double s = 0.0;
      for (int jj = 0; jj < m; ++jj) s = fma(A[(int64_t)(k + 1 + jj) * ld + i], v[jj], s);
      w[i] = s;
    }
    __syncthreads();
    for (int e = tid; e < n * m; e += bd) {
      const int i = e % n, jj = e / n;
      A[(int64_t)(k + 1 + jj) * ld + i] -= t * w[i] * v[jj];
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) tau[k] = 0.0;
  }
}

// Symmetric A (n x n, ld, both triangles stored) <- Q^T A Q tridiagonal, with
// the same reflector storage as k_hessenberg (v below the subdiagonal of
// column k, tau[k]).  Per step: p = tau A22 v, w = p - (tau/2)(p.v) v,
// A22 -= v w^T + w v^T.  One CTA; shared memory 3n + 32 doubles.
__global__ void k_sytrd(int n, double* A, int ld, double* tau) {
  extern __shared__ double sm[];
  double* v = sm;
  double* w = sm + n;
  double* red = sm + 2 * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = A + (int64_t)k * ld + (k + 1);
    double loc = 0.0;
    for (int i = 1 + tid; i < m; i += bd) loc += x[i] * x[i];
    const double sig = block_sum(loc, red);
    const double alpha = x[0];
    if (sig == 0.0) {
      if (tid == 0) tau[k] = 0.0;
      __syncthreads();
      continue;
    }
    const double nrm = sqrt(alpha * alpha + sig);
    const double beta = alpha <= 0.0 ? nrm : -nrm;
    const double t = (beta - alpha) / beta;
    const double sc = 1.0 / (alpha - beta);
    for (int i = tid; i < m; i += bd) v[i] = (i == 0) ? 1.0 : x[i] * sc;
    __syncthreads();
    for (int i = 1 + tid; i < m; i += bd) x[i] = v[i];
    if (tid == 0) {
      x[0] = beta;
      A[k + (int64_t)(k + 1) * ld] = beta;
      tau[k] = t;
    }
    // p = tau * A22 v (A22 symmetric: use its columns)
    for (int j = tid; j < m; j += bd) {
      const double* col = A + (int64_t)(k + 1 + j) * ld + (k + 1);
      double s = 0.0;
      for (int i = 0; i < m; ++i) s = fma(col[i], v[i], s);
      w[j] = t * s;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = tid; i < m; i += bd) pv += w[i] * v[i];
    pv = block_sum(pv, red);
    for (int i = tid; i < m; i += bd) w[i] -= 0.5 * t * pv * v[i];
    __syncthreads();
    for (int e = tid; e < m * m; e += bd) {
      const int i = e % m, j = e / m;
      A[(int64_t)(k + 1 + j) * ld + (k + 1 + i)] -= v[i] * w[j] + w[i] * v[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) tau[k] = 0.0;
  }
}

// y <- Q y for every column of Y (n x nvec, ld), Q = H_0 ... H_{n-3} from
// k_hessenberg's storage in A.  One CTA per column.
__global__ void k_apply_q(int n, const double* __restrict__ A, int lda, const double* __restrict__ tau,
                          double* __restrict__ Y, int ldy) {
  __shared__ double red[32];
  double* y = Y + (int64_t)blockIdx.x * ldy;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int k = n - 3; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;
    const int m = n - k - 1;
    const double* vs = A + (int64_t)k * lda + (k + 1);
    double loc = 0.0;
    for (int i = tid; i < m; i += bd) loc += (i == 0 ? 1.0 : vs[i]) * y[k + 1 + i];
    const double s = block_sum(loc, red) * t;
    for (int i = tid; i < m; i += bd) y[k + 1 + i] -= s * (i == 0 ? 1.0 : vs[i]);
    __syncthreads();
  }
}

// ------------------------------------------------------- Francis QR

template <class Real>
__device__ __forceinline__ void two_by_two_eigs(Real a, Real b, Real c, Real d, double& r1, double& i1, double& r2,
                                                double& i2) {
  const Real p = Real(0.5) * (a - d);
  const Real bc = b * c;
  const Real disc = p * p + bc;
  if (disc >= Real(0)) {
    const Real z = p + copysign(sqrt(disc), p);
    r1 = (double)(d + z);
    r2 = (z != Real(0)) ? (double)(d - bc / z) : (double)(d + z);
    i1 = i2 = 0.0;
  } else {
    const Real re = d + p, im = sqrt(-disc);
    r1 = r2 = (double)re;
    i1 = (double)im;
    i2 = -(double)im;
  }
}

template <class Real>
struct EpsOf;
template <>
struct EpsOf<float> {
  static constexpr float v = FLT_EPSILON;
};

// Eigenvalues of the upper Hessenberg matrix Hin (n x n, ld; FP64) by Francis
// double-shift QR in precision Real.  One warp; the matrix is copied into
// shared memory (leading dimension ldw, odd so that a warp's row accesses hit
// distinct banks) when kSmem, otherwise into the global scratch.  With
// Real = float this only supplies starting shifts: every eigenvalue is then
// refined in FP64 by k_hess_rqi.  Matrices that fit in shared memory take the
// multishift kernel k_hqr_ms instead; this one serves larger n from global
// scratch.
constexpr int kHqrT = 5;   // rows per lane per batch of the column update (160 per warp)

// kSmem: the matrix lives in shared memory, addressed as such with 32-bit
// indices (a pointer that may point to either space compiles to generic
// loads and stores, which made every bulge step about twice as slow).
template <class Real, bool kSmem>
__global__ void k_hqr(int n, const double* __restrict__ Hin, int ldh, double* wr, double* wi, Real* Hscratch,
                      int32_t* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Idx = typename std::conditional<kSmem, int, int64_t>::type;
  const int ldw = n | 1;
  Real* H = kSmem ? reinterpret_cast<Real*>(smem_raw) : Hscratch;
  const int lane = threadIdx.x;
  // Deflation threshold.  These eigenvalues only seed the FP64
  // Rayleigh-quotient refinement: an eigenvalue deflated at a subdiagonal of
  // 1e-5 (relative) is already accurate to about its square, which the
  // refinement takes to FP64 accuracy in its first step; waiting for FP32
  // roundoff would cost about one more QR sweep per eigenvalue.
  const Real deflate = fmax(EpsOf<Real>::v, Real(1e-5));
  // copy (Hessenberg part, zeros below) and the max-abs norm, lanes over rows
  Real amax = 0;
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    for (int i = lane; i < n; i += 32) {
      const Real v = (i <= j + 1) ? (Real)Hin[i + (int64_t)j * ldh] : Real(0);
      H[(Idx)i + (Idx)j * (Idx)ldw] = v;
      amax = fmax(amax, fabs(v));
    }
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  __syncwarp();
#define HH(i, j) H[(Idx)(i) + (Idx)(j) * (Idx)ldw]
  Real anorm = amax;
  if (anorm == Real(0)) anorm = 1;
  int hi = n - 1, its = 0, total = 0;
  while (hi >= 0) {
    int lo = hi;
    while (lo > 0) {
      Real s = fabs(HH(lo - 1, lo - 1)) + fabs(HH(lo, lo));
      if (s == Real(0)) s = anorm;
      if (fabs(HH(lo, lo - 1)) <= deflate * s) break;
      --lo;
    }
    if (lo > 0) {
      __syncwarp();
      if (lane == 0) HH(lo, lo - 1) = 0;
      __syncwarp();
    }
    if (lo == hi) {
      if (lane == 0) {
        wr[hi] = (double)HH(hi, hi);
        wi[hi] = 0.0;
      }
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {
      double r1, i1, r2, i2;
      two_by_two_eigs<Real>(HH(hi - 1, hi - 1), HH(hi - 1, hi), HH(hi, hi - 1), HH(hi, hi), r1, i1, r2, i2);
      if (lane == 0) {
        wr[hi - 1] = r1;
        wi[hi - 1] = i1;
        wr[hi] = r2;
        wi[hi] = i2;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (its >= 90) {
      if (lane == 0) {
        raise_status(info, DMD_ENUMERIC, 3000 + hi);
        for (int i = 0; i <= hi; ++i) wr[i] = wi[i] = nan("");
      }
      return;
    }
    ++its;
    ++total;
    // double shift from the trailing 2x2 block (sum s, product t); exceptional every 10 sweeps
    Real s, t;
    if (its % 10 == 0) {
      const Real w = fabs(HH(hi, hi - 1)) + fabs(HH(hi - 1, hi - 2));
      const Real h = Real(0.75) * w + HH(hi, hi);
      s = Real(2) * h;
      t = h * h + Real(0.4375) * w * w;
    } else {
      s = HH(hi - 1, hi - 1) + HH(hi, hi);
      t = HH(hi - 1, hi - 1) * HH(hi, hi) - HH(hi - 1, hi) * HH(hi, hi - 1);
    }
    Real x = HH(lo, lo) * HH(lo, lo) + HH(lo, lo + 1) * HH(lo + 1, lo) - s * HH(lo, lo) + t;
    Real y = HH(lo + 1, lo) * (HH(lo, lo) + HH(lo + 1, lo + 1) - s);
    Real z = HH(lo + 1, lo) * HH(lo + 2, lo + 1);
    for (int k = lo; k <= hi - 2; ++k) {
      // reflector P = I - tau v v^T, v = [1, v1, v2], P [x y z]^T = [beta 0 0]^T
      const Real nrm = sqrt(x * x + y * y + z * z);
      if (nrm != Real(0) && (y != Real(0) || z != Real(0))) {
        // fast division: these eigenvalues only seed the FP64 refinement
        const Real beta = x <= Real(0) ? nrm : -nrm;
        const Real tau = __fdividef(beta - x, beta);
        const Real sc = __fdividef(Real(1), x - beta);
        const Real v1 = y * sc, v2 = z * sc;
        const int c0 = max(lo, k - 1);
        // row update, batched like the column update below: every lane loads
        // its columns' three entries first so the shared-memory latencies
        // overlap, then updates them
        for (int cb = c0; cb <= hi; cb += 32 * kHqrT) {
          Real r0[kHqrT], r1[kHqrT], r2[kHqrT];
#pragma unroll
          for (int t = 0; t < kHqrT; ++t) {
            const int c = cb + lane + 32 * t;
            r0[t] = c <= hi ? HH(k, c) : Real(0);
            r1[t] = c <= hi ? HH(k + 1, c) : Real(0);
            r2[t] = c <= hi ? HH(k + 2, c) : Real(0);
          }
#pragma unroll
          for (int t = 0; t < kHqrT; ++t) {
            const int c = cb + lane + 32 * t;
            const Real p = tau * (r0[t] + v1 * r1[t] + v2 * r2[t]);
            if (c <= hi) {
              HH(k, c) = r0[t] - p;
              HH(k + 1, c) = r1[t] - p * v1;
              HH(k + 2, c) = r2[t] - p * v2;
            }
          }
        }
        __syncwarp();
        if (k > lo && lane == 0) {
          HH(k + 1, k - 1) = 0;
          HH(k + 2, k - 1) = 0;
        }
        const int rend = min(k + 3, hi);
        // column update: every lane loads all of its rows first (their
        // shared-memory latencies overlap); rows lo..k+3 usually span most
        // of the window, so five per lane are rarely wasted
        for (int rb = lo; rb <= rend; rb += 32 * kHqrT) {
          Real q0[kHqrT], q1[kHqrT], q2[kHqrT];
#pragma unroll
          for (int t = 0; t < kHqrT; ++t) {
            const int rr = rb + lane + 32 * t;
            q0[t] = rr <= rend ? HH(rr, k) : Real(0);
            q1[t] = rr <= rend ? HH(rr, k + 1) : Real(0);
            q2[t] = rr <= rend ? HH(rr, k + 2) : Real(0);
          }
#pragma unroll
          for (int t = 0; t < kHqrT; ++t) {
            const int rr = rb + lane + 32 * t;
            const Real p = tau * (q0[t] + v1 * q1[t] + v2 * q2[t]);
            if (rr <= rend) {
              HH(rr, k) = q0[t] - p;
              HH(rr, k + 1) = q1[t] - p * v1;
              HH(rr, k + 2) = q2[t] - p * v2;
            }
          }
        }
        __syncwarp();
      }
      x = HH(k + 1, k);
      y = HH(k + 2, k);
      if (k < hi - 2) z = HH(k + 3, k);
    }
    // final 2-vector reflector on rows/columns hi-1, hi
    {
      const Real nrm = sqrt(x * x + y * y);
      if (nrm != Real(0) && y != Real(0)) {
        const Real beta = x <= Real(0) ? nrm : -nrm;
        const Real tau = __fdividef(beta - x, beta);
        const Real v1 = __fdividef(y, x - beta);
        const int k = hi - 1;
        for (int c = max(lo, k - 1) + lane; c <= hi; c += 32) {
          const Real p = tau * (HH(k, c) + v1 * HH(k + 1, c));
          HH(k, c) -= p;
          HH(k + 1, c) -= p * v1;
        }
        __syncwarp();
        if (k > lo && lane == 0) HH(k + 1, k - 1) = 0;
        for (int rr = lo + lane; rr <= hi; rr += 32) {
          const Real p = tau * (HH(rr, k) + v1 * HH(rr, k + 1));
          HH(rr, k) -= p;
          HH(rr, k + 1) -= p * v1;
        }
        __syncwarp();
      }
    }
  }
#undef HH
  if (lane == 0 && info) info[3] = total;
}

// --------------------------------------------- Francis QR, multishift chain

// FP32 eigenvalue estimates of an unreduced Hessenberg window by chains of
// small bulges (the small-bulge multishift form of Francis' algorithm): each
// sweep of a wide window takes 2 s shifts, the eigenvalues of its trailing
// 2s x 2s block, and chases s double-shift bulges down the window together,
// three rows apart, one warp per bulge.  A chain step forms every bulge's
// reflector from the current matrix, applies them from the left (disjoint
// row triples), then from the right (disjoint column triples), with a CTA
// barrier between the two: the same similarity as chasing the bulges one
// after the other (left and right products commute, and no reflector reads
// an entry another bulge of the same step writes).  A step costs about what
// one double-shift step costs, so a sweep applies s times the shifts.  The
// kernel is bound by the latency of each warp's instruction stream
// (measured: ~6 cycles per issued instruction, one warp per scheduler), so
// the step is written for few instructions (compile-time strides, one
// reciprocal square root for the norm); splitting a bulge over two warps
// was measured slower (more barrier waits).
// Narrow windows, every 10th sweep of a window (exceptional shifts) and
// windows whose shift problem does not converge take one double-shift sweep.
constexpr int kMsBulges = 4;   // bulges per chain
constexpr int kMsSplit = 1;    // warps per bulge
constexpr int kMsWarps = kMsBulges * kMsSplit;
constexpr int kMsMin = 40;     // narrower windows take double-shift sweeps
constexpr int kMsLd = 2 * kMsBulges + 1;

// P = I - tau v v^T, v = (1, v1, v2), with P (x, y, z)^T = (beta, 0, 0)^T;
// tau = 0 when there is nothing to annihilate.  Fast divisions: these
// eigenvalues only seed the FP64 refinement.
struct Refl3 {
  float tau, v1, v2;
};
__device__ __forceinline__ Refl3 refl3(float x, float y, float z) {
  Refl3 P{0.f, 0.f, 0.f};
  const float n2 = x * x + y * y + z * z;
  if (n2 > 0.f && (y != 0.f || z != 0.f)) {
    const float nrm = n2 * rsqrtf(n2);
    const float beta = x <= 0.f ? nrm : -nrm;
    P.tau = __fdividef(beta - x, beta);
    const float sc = __fdividef(1.f, x - beta);
    P.v1 = y * sc;
    P.v2 = z * sc;
  }
  return P;
}

// Rows k .. k + nr - 1 (nr = 2 or 3) of H (column-major, ld ldw) times P,
// columns c0 .. c1, by `parts` warps (this one is part `part`): element e of
// the range goes to lane e % 32 of part (e / 32) % parts, one element after
// the other (a rolled loop: fewer instructions than batched loads with
// per-slot guards, which the instruction-latency-bound step pays for).  Column
// zc (the bulge just annihilated; -1 for none) gets exact zeros below row k.
template <int PARTS>
__device__ __forceinline__ void ms_rows(float* H, int ldw, int k, int nr, int c0, int c1, Refl3 P, int zc,
                                        int lane, int part) {
  constexpr int stride = 32 * PARTS;
  float* h0 = H + k;
#pragma unroll 1
  for (int c = c0 + part * 32 + lane; c <= c1; c += stride) {
    float* hc = h0 + c * ldw;
    const float r0 = hc[0], r1 = hc[1], r2 = nr == 3 ? hc[2] : 0.f;
    const float p = P.tau * (r0 + P.v1 * r1 + P.v2 * r2);
    hc[0] = r0 - p;
    hc[1] = c == zc ? 0.f : r1 - p * P.v1;
    if (nr == 3) hc[2] = c == zc ? 0.f : r2 - p * P.v2;
  }
}

// Columns k .. k + nr - 1 of H times P, rows r0 .. r1, by `parts` warps.
template <int PARTS>
__device__ __forceinline__ void ms_cols(float* H, int ldw, int k, int nr, int r0, int r1, Refl3 P, int lane,
                                        int part) {
  constexpr int stride = 32 * PARTS;
  float* c0p = H + k * ldw;
#pragma unroll 1
  for (int r = r0 + part * 32 + lane; r <= r1; r += stride) {
    const float q0 = c0p[r], q1 = c0p[r + ldw], q2 = nr == 3 ? c0p[r + 2 * ldw] : 0.f;
    const float p = P.tau * (q0 + P.v1 * q1 + P.v2 * q2);
    c0p[r] = q0 - p;
    c0p[r + ldw] = q1 - p * P.v1;
    if (nr == 3) c0p[r + 2 * ldw] = q2 - p * P.v2;
  }
}

// First column of (H - s1)(H - s2) at the top of window [lo, hi] (s = s1 + s2,
// t = s1 s2), rows lo .. lo + 2.
__device__ __forceinline__ void ms_intro(const float* H, int ldw, int lo, float s, float t, float& x, float& y,
                                         float& z) {
  const float h00 = H[lo + lo * ldw], h01 = H[lo + (lo + 1) * ldw], h10 = H[lo + 1 + lo * ldw];
  const float h11 = H[lo + 1 + (lo + 1) * ldw], h21 = H[lo + 2 + (lo + 1) * ldw];
  x = h00 * h00 + h01 * h10 - s * h00 + t;
  y = h10 * (h00 + h11 - s);
  z = h10 * h21;
}

// One double-shift sweep over window [lo, hi] (hi - lo >= 2) by one warp.
__device__ void ms_double_sweep(float* H, int ldw, int lo, int hi, float s, float t, int lane) {
  float x, y, z;
  ms_intro(H, ldw, lo, s, t, x, y, z);
  for (int k = lo; k <= hi - 1; ++k) {
    const int nr = k <= hi - 2 ? 3 : 2;
    if (k > lo) {
      x = H[k + (k - 1) * ldw];
      y = H[k + 1 + (k - 1) * ldw];
      z = nr == 3 ? H[k + 2 + (k - 1) * ldw] : 0.f;
    }
    const Refl3 P = refl3(x, y, nr == 3 ? z : 0.f);
    if (P.tau != 0.f) {
      ms_rows<1>(H, ldw, k, nr, max(lo, k - 1), hi, P, k > lo ? k - 1 : -1, lane, 0);
      __syncwarp();
      ms_cols<1>(H, ldw, k, nr, lo, min(k + 3, hi), P, lane, 0);
      __syncwarp();
    }
  }
}

// Bottom of window [lo, hi]: the largest lo <= hi with H(lo, lo-1)
// negligible relative to its diagonal neighbours (0 if none), i.e. the
// first such subdiagonal scanning up from hi; the lanes of a warp test 32
// subdiagonals at once (every lane gets the answer).
__device__ __forceinline__ int ms_scan(const float* H, int ldw, int hi, float deflate, float anorm, int lane) {
  for (int top = hi; top > 0; top -= 32) {
    const int i = top - lane;
    bool small = false;
    if (i > 0) {
      float s = fabsf(H[i - 1 + (i - 1) * ldw]) + fabsf(H[i + i * ldw]);
      if (s == 0.f) s = anorm;
      small = fabsf(H[i + (i - 1) * ldw]) <= deflate * s;
    }
    const unsigned m = __ballot_sync(0xffffffffu, small);
    if (m) return top - (__ffs(m) - 1);
  }
  return 0;
}

// Standard double shift of window [lo, hi] (sum s, product t): the trailing
// 2 x 2 block, or every 10th sweep the exceptional shift.
__device__ __forceinline__ void ms_shift(const float* H, int ldw, int hi, int its, float& s, float& t) {
  if (its % 10 == 0) {
    const float w = fabsf(H[hi + (hi - 1) * ldw]) + fabsf(H[hi - 1 + (hi - 2) * ldw]);
    const float h = 0.75f * w + H[hi + hi * ldw];
    s = 2.f * h;
    t = h * h + 0.4375f * w * w;
  } else {
    const float a = H[hi - 1 + (hi - 1) * ldw], b = H[hi - 1 + hi * ldw], c = H[hi + (hi - 1) * ldw],
                d = H[hi + hi * ldw];
    s = a + d;
    t = a * d - b * c;
  }
}

// Eigenvalues of the k x k Hessenberg matrix A (ld lda, overwritten) by
// double-shift sweeps, one warp; er / ei written by lane 0 (conjugate pairs
// adjacent).  false when a window needs more than 30 sweeps.
__device__ bool ms_small_eigs(float* A, int lda, int k, float* er, float* ei, int lane) {
  float anorm = 0.f;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) anorm = fmaxf(anorm, fabsf(A[i + j * lda]));
  if (anorm == 0.f) anorm = 1.f;
  int hi = k - 1, its = 0;
  while (hi >= 0) {
    __syncwarp();
    const int lo = ms_scan(A, lda, hi, 1e-5f, anorm, lane);
    __syncwarp();
    if (lo > 0 && lane == 0) A[lo + (lo - 1) * lda] = 0.f;
    if (lo == hi) {
      if (lane == 0) {
        er[hi] = A[hi + hi * lda];
        ei[hi] = 0.f;
      }
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {
      double r1, i1, r2, i2;
      two_by_two_eigs<float>(A[hi - 1 + (hi - 1) * lda], A[hi - 1 + hi * lda], A[hi + (hi - 1) * lda],
                             A[hi + hi * lda], r1, i1, r2, i2);
      if (lane == 0) {
        er[hi - 1] = (float)r1;
        ei[hi - 1] = (float)i1;
        er[hi] = (float)r2;
        ei[hi] = (float)i2;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (its >= 30) return false;
    ++its;
    float s, t;
    ms_shift(A, lda, hi, its, s, t);
    __syncwarp();
    ms_double_sweep(A, lda, lo, hi, s, t, lane);
  }
  __syncwarp();
  return true;
}

__global__ void __launch_bounds__(32 * kMsWarps, 1)
    k_hqr_ms(int n, const double* __restrict__ Hin, int ldh, double* wr, double* wi, int32_t* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldw = n | 1;
  float* H = reinterpret_cast<float*>(smem_raw);
  float* Hs = H + n * ldw;               // the trailing block whose eigenvalues are the shifts
  float* ser = Hs + 2 * kMsBulges * kMsLd;
  float* sei = ser + 2 * kMsBulges;
  float* bs = sei + 2 * kMsBulges;       // per bulge: shift sum and product
  float* bt = bs + kMsBulges;
  float* red = bt + kMsBulges;           // [kMsWarps]
  int* nbulge = reinterpret_cast<int*>(red + kMsWarps);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float deflate = fmaxf(FLT_EPSILON, 1e-5f);   // as k_hqr: these eigenvalues seed the FP64 refinement
  float amax = 0.f;
  for (int j = 0; j < n; ++j)
    for (int i = tid; i < n; i += blockDim.x) {
      const float v = (i <= j + 1) ? (float)Hin[i + (int64_t)j * ldh] : 0.f;
      H[i + j * ldw] = v;
      amax = fmaxf(amax, fabsf(v));
    }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (lane == 0) red[warp] = amax;
  __syncthreads();
  float anorm = 0.f;
  for (int w = 0; w < kMsWarps; ++w) anorm = fmaxf(anorm, red[w]);
  if (anorm == 0.f) anorm = 1.f;
  int hi = n - 1, its = 0, total = 0;
  while (hi >= 0) {
    __syncthreads();
    const int lo = ms_scan(H, ldw, hi, deflate, anorm, lane);   // every warp, the same answer
    __syncthreads();
    if (lo > 0 && tid == 0) H[lo + (lo - 1) * ldw] = 0.f;
    if (lo == hi) {
      if (tid == 0) {
        wr[hi] = (double)H[hi + hi * ldw];
        wi[hi] = 0.0;
      }
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {
      double r1, i1, r2, i2;
      two_by_two_eigs<float>(H[hi - 1 + (hi - 1) * ldw], H[hi - 1 + hi * ldw], H[hi + (hi - 1) * ldw],
                             H[hi + hi * ldw], r1, i1, r2, i2);
      if (tid == 0) {
        wr[hi - 1] = r1;
        wi[hi - 1] = i1;
        wr[hi] = r2;
        wi[hi] = i2;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (its >= 90) {
      if (tid == 0) {
        raise_status(info, DMD_ENUMERIC, 3000 + hi);
        for (int i = 0; i <= hi; ++i) wr[i] = wi[i] = nan("");
      }
      return;
    }
    ++its;
    ++total;
    int s = 1;
    if (hi - lo + 1 >= kMsMin && its % 10 != 0) {
      // 2 s shifts: eigenvalues of the trailing 2s x 2s block, paired per bulge
      constexpr int k2 = 2 * kMsBulges;
      if (warp == 0) {
        for (int e = lane; e < k2 * k2; e += 32) {
          const int i = e % k2, j = e / k2;
          Hs[i + j * kMsLd] = i <= j + 1 ? H[hi - k2 + 1 + i + (hi - k2 + 1 + j) * ldw] : 0.f;
        }
        __syncwarp();
        const bool ok = ms_small_eigs(Hs, kMsLd, k2, ser, sei, lane);
        if (lane == 0) {
          int nb = 0;
          float pend = 0.f;
          bool have = false;
          for (int i = 0; ok && i < k2;) {
            if (sei[i] != 0.f) {   // a conjugate pair (adjacent)
              bs[nb] = 2.f * ser[i];
              bt[nb] = ser[i] * ser[i] + sei[i] * sei[i];
              ++nb;
              i += 2;
            } else if (have) {     // two real shifts
              bs[nb] = pend + ser[i];
              bt[nb] = pend * ser[i];
              ++nb;
              have = false;
              ++i;
            } else {
              pend = ser[i];
              have = true;
              ++i;
            }
          }
          *nbulge = (ok && nb == kMsBulges) ? nb : 1;
        }
      }
      __syncthreads();
      s = *nbulge;
    }
    if (s > 1) {
      const int T = (hi - 1 - lo) + 3 * (s - 1) + 1;
      const int bulge = warp / kMsSplit, part = warp % kMsSplit;
      for (int t = 0; t < T; ++t) {
        const int k = lo + t - 3 * bulge;
        const bool act = bulge < s && k >= lo && k <= hi - 1;
        const int nr = k <= hi - 2 ? 3 : 2;
        Refl3 P{0.f, 0.f, 0.f};
        if (act) {
          float x, y, z;
          if (k == lo) {
            ms_intro(H, ldw, lo, bs[bulge], bt[bulge], x, y, z);
          } else {
            x = H[k + (k - 1) * ldw];
            y = H[k + 1 + (k - 1) * ldw];
            z = nr == 3 ? H[k + 2 + (k - 1) * ldw] : 0.f;
          }
          P = refl3(x, y, nr == 3 ? z : 0.f);
          if (P.tau != 0.f)
            ms_rows<kMsSplit>(H, ldw, k, nr, max(lo, k - 1), hi, P, k > lo ? k - 1 : -1, lane, part);
        }
        __syncthreads();
        if (act && P.tau != 0.f) ms_cols<kMsSplit>(H, ldw, k, nr, lo, min(k + 3, hi), P, lane, part);
        __syncthreads();
      }
    } else if (warp == 0) {
      float sh, th;
      ms_shift(H, ldw, hi, its, sh, th);
      ms_double_sweep(H, ldw, lo, hi, sh, th, lane);
    }
  }
  if (tid == 0 && info) info[3] = total;
}

// ---------------------------------------------- inverse iteration (Hessenberg)

// Rayleigh-quotient inverse iteration on the FP64 Hessenberg matrix for each
// head eigenvalue estimate mu = wr + i wi (wi >= 0): factor H - mu I (LU with
// pivoting between adjacent rows, O(n^2)), solve y = (H - mu I)^{-1} x,
// update mu <- mu + (x^H x) / (x^H y) and x <- y / |y|.  Three iterations
// take an FP32-accurate estimate to FP64 accuracy (quadratic convergence);
// a correction larger than 1e-3 |mu| is not applied (the shift then stays
// put, so the iteration cannot wander to another eigenvalue).  Writes the
// refined eigenvalue (and its conjugate partner, index e + 1) and the
// eigenvector y of H.  One CTA per head; work: 2 n^2 doubles per CTA.
__global__ void k_hess_rqi(int n, const double* __restrict__ H, int ldh, double* __restrict__ wr,
                           double* __restrict__ wi, const int* __restrict__ heads, double* __restrict__ Yre,
                           double* __restrict__ Yim, double* __restrict__ work, const double* __restrict__ hnorm_ptr) {
  extern __shared__ double sm[];
  double* mre = sm;                 // multipliers
  double* mim = sm + n;
  double* xre = sm + 2 * n;
  double* xim = sm + 3 * n;
  double* yre = sm + 4 * n;
  double* yim = sm + 5 * n;
  int* piv = reinterpret_cast<int*>(sm + 6 * n);
  __shared__ double red[32];
  __shared__ double mu_s[2];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int e = heads[blockIdx.x];
  if (e < 0) return;   // padding beyond the actual number of heads
  double mur = wr[e], mui = wi[e];
  const bool pair = mui > 0.0;
  double* Ur = work + (int64_t)blockIdx.x * 2 * n * n;
  double* Ui = Ur + (int64_t)n * n;
#define UR(i, j) Ur[(i) + (int64_t)(j) * n]
#define UI(i, j) Ui[(i) + (int64_t)(j) * n]
  const double hnorm = fmax(*hnorm_ptr, DBL_MIN);
  const double tiny = kEps * hnorm;
  for (int i = tid; i < n; i += bd) {
    xre[i] = 1.0 / sqrt((double)n);
    xim[i] = 0.0;
  }
  for (int it = 0; it < 3; ++it) {
    __syncthreads();
    for (int q = tid; q < n * n; q += bd) {
      const int i = q % n, j = q / n;
      double hr = (i <= j + 1) ? H[i + (int64_t)j * ldh] : 0.0, hi_ = 0.0;
      if (i == j) {
        hr -= mur;
        hi_ = -mui;
      }
      UR(i, j) = hr;
      UI(i, j) = hi_;
    }
    __syncthreads();
    for (int k = 0; k + 1 < n; ++k) {
      if (tid == 0) {
        const double ar = UR(k, k), ai = UI(k, k), br = UR(k + 1, k), bi = UI(k + 1, k);
        const bool sw = (br * br + bi * bi) > (ar * ar + ai * ai);
        piv[k] = sw ? 1 : 0;
        double pr = sw ? br : ar, pi = sw ? bi : ai;
        double orr = sw ? ar : br, oi = sw ? ai : bi;
        if (pr == 0.0 && pi == 0.0) pr = tiny;
        const double den = pr * pr + pi * pi;
        mre[k] = (orr * pr + oi * pi) / den;
        mim[k] = (oi * pr - orr * pi) / den;
        UR(k, k) = pr;
        UI(k, k) = pi;
      }
      __syncthreads();
      const int sw = piv[k];
      const double lr = mre[k], li = mim[k];
      for (int j = k + 1 + tid; j < n; j += bd) {
        double ar = UR(k, j), ai = UI(k, j), br = UR(k + 1, j), bi = UI(k + 1, j);
        if (sw) {
          const double tr = ar, ti = ai;
          ar = br;
          ai = bi;
          br = tr;
          bi = ti;
        }
        UR(k, j) = ar;
        UI(k, j) = ai;
        UR(k + 1, j) = br - (lr * ar - li * ai);
        UI(k + 1, j) = bi - (lr * ai + li * ar);
      }
      __syncthreads();
    }
    if (tid == 0 && UR(n - 1, n - 1) == 0.0 && UI(n - 1, n - 1) == 0.0) UR(n - 1, n - 1) = tiny;
    // y = P L^{-1} x (forward, sequential), then U y = that (back substitution)
    if (tid == 0) {
      for (int i = 0; i < n; ++i) {
        yre[i] = xre[i];
        yim[i] = xim[i];
      }
      for (int k = 0; k + 1 < n; ++k) {
        if (piv[k]) {
          const double tr = yre[k], ti = yim[k];
          yre[k] = yre[k + 1];
          yim[k] = yim[k + 1];
          yre[k + 1] = tr;
          yim[k + 1] = ti;
        }
        const double lr = mre[k], li = mim[k];
        yre[k + 1] -= lr * yre[k] - li * yim[k];
        yim[k + 1] -= lr * yim[k] + li * yre[k];
      }
    }
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {
      double sr = 0.0, si = 0.0;
      for (int j = i + 1 + tid; j < n; j += bd) {
        const double ur = UR(i, j), ui = UI(i, j);
        sr += ur * yre[j] - ui * yim[j];
        si += ur * yim[j] + ui * yre[j];
      }
      sr = block_sum(sr, red);
      si = block_sum(si, red);
      if (tid == 0) {
        const double br = yre[i] - sr, bi = yim[i] - si;
        const double ur = UR(i, i), ui = UI(i, i), den = ur * ur + ui * ui;
        yre[i] = (br * ur + bi * ui) / den;
        yim[i] = (bi * ur - br * ui) / den;
      }
      __syncthreads();
    }
    // Rayleigh quotient: theta = x^H y (x has unit norm); mu += 1 / theta
    double tr_ = 0.0, ti_ = 0.0, yy = 0.0;
    for (int i = tid; i < n; i += bd) {
      tr_ += xre[i] * yre[i] + xim[i] * yim[i];
      ti_ += xre[i] * yim[i] - xim[i] * yre[i];
      yy += yre[i] * yre[i] + yim[i] * yim[i];
    }
    tr_ = block_sum(tr_, red);
    ti_ = block_sum(ti_, red);
    yy = block_sum(yy, red);
    if (tid == 0) {
      const double den = tr_ * tr_ + ti_ * ti_;
      double dr = 0.0, di = 0.0;
      if (den > 0.0 && isfinite(den)) {
        dr = tr_ / den;
        di = -ti_ / den;
      }
      const double mag = hypot(mur, mui);
      if (hypot(dr, di) < 1e-3 * fmax(mag, 1e-300)) {
        mur += dr;
        if (pair) mui += di;   // a real eigenvalue stays real
      }
      mu_s[0] = mur;
      mu_s[1] = mui;
    }
    const double inv = (yy > 0.0 && isfinite(yy)) ? 1.0 / sqrt(yy) : 1.0;
    __syncthreads();
    mur = mu_s[0];
    mui = mu_s[1];
    for (int i = tid; i < n; i += bd) {
      xre[i] = yre[i] * inv;
      xim[i] = yim[i] * inv;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += bd) {
    Yre[i + (int64_t)blockIdx.x * n] = xre[i];
    Yim[i + (int64_t)blockIdx.x * n] = xim[i];
  }
  if (tid == 0) {
    wr[e] = mur;
    wi[e] = pair ? mui : 0.0;
    if (pair && e + 1 < n) {
      wr[e + 1] = mur;
      wi[e + 1] = -mui;
    }
  }
#undef UR
#undef UI
}

// Unit 2-norm, largest-magnitude entry real positive.  One CTA per column.
// The same Rayleigh-quotient inverse iteration (same shift rule, same
// outputs) with one warp per head and U in shared memory: no block barriers,
// no global round trips.  LU of the Hessenberg H - mu I row by row: an active
// row a (U's row k once the adjacent-row pivot is taken) and the next matrix
// row h; U is stored row-packed (row k holds columns k..n-1 at offset
// k n - k (k - 1) / 2).  The back substitution is column-oriented (no
// reductions).  Shared memory: n (n + 1) + 8 n doubles + n ints.
__global__ void __launch_bounds__(32) k_hess_rqi_w(int n, const double* __restrict__ H, int ldh,
                                                   double* __restrict__ wr, double* __restrict__ wi,
                                                   const int* __restrict__ heads, double* __restrict__ Yre,
                                                   double* __restrict__ Yim, const double* __restrict__ hnorm_ptr) {
  extern __shared__ double sm[];
  const int np = n * (n + 1) / 2;
  double* Ur = sm;
  double* Ui = Ur + np;
  double* ar = Ui + np;     // active row (columns k..)
  double* ai = ar + n;
  double* mre = ai + n;     // multipliers
  double* mim = mre + n;
  double* xre = mim + n;
  double* xim = xre + n;
  double* yre = xim + n;
  double* yim = yre + n;
  int* piv = reinterpret_cast<int*>(yim + n);
  const int lane = threadIdx.x;
  const int e = heads[blockIdx.x];
  if (e < 0) return;
  double mur = wr[e], mui = wi[e];
  const bool pair = mui > 0.0;
  const double tiny = kEps * fmax(*hnorm_ptr, DBL_MIN);
  auto off = [n](int k) { return k * n - k * (k - 1) / 2; };
  for (int i = lane; i < n; i += 32) {
    xre[i] = 1.0 / sqrt((double)n);
    xim[i] = 0.0;
  }
  for (int it = 0; it < 3; ++it) {
    // active row = row 0 of H - mu I
    for (int j = lane; j < n; j += 32) {
      ar[j] = H[(int64_t)j * ldh] - (j == 0 ? mur : 0.0);
      ai[j] = j == 0 ? -mui : 0.0;
    }
    __syncwarp();
    // row k + 1 of H at columns k + lane + 32 t, loaded one step ahead
    constexpr int kMaxT = 5;   // n <= 160
    double hrow[kMaxT];
#pragma unroll
    for (int t = 0; t < kMaxT; ++t) {
      const int j = lane + 32 * t;
      hrow[t] = (n > 1 && j < n) ? H[1 + (int64_t)j * ldh] : 0.0;
    }
    for (int k = 0; k + 1 < n; ++k) {
      // next row of H - mu I (columns k.. ; Hessenberg: zero left of k)
      const double hkr = __shfl_sync(0xffffffffu, hrow[0], 0);
      const double pa = ar[k] * ar[k] + ai[k] * ai[k];
      const bool sw = hkr * hkr > pa;
      // pivot p and the other entry o of column k; multiplier l = o / p
      double pr = sw ? hkr : ar[k], pim = sw ? 0.0 : ai[k];
      const double orr = sw ? ar[k] : hkr, oi = sw ? ai[k] : 0.0;
      if (pr == 0.0 && pim == 0.0) pr = tiny;
      const double iden = rcp_nr(pr * pr + pim * pim);
      const double lr = (orr * pr + oi * pim) * iden, li = (oi * pr - orr * pim) * iden;
      double* ur = Ur + off(k) - k;   // ur[j] = U(k, j)
      double* ui = Ui + off(k) - k;
      double hnext[kMaxT];
#pragma unroll
      for (int t = 0; t < kMaxT; ++t) {
        const int j = k + 1 + lane + 32 * t;
        hnext[t] = (k + 2 < n && j < n) ? H[(k + 2) + (int64_t)j * ldh] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < kMaxT; ++t) {
        const int j = k + lane + 32 * t;
        if (j >= n) break;
        double hr = hrow[t], hi = 0.0;
        if (j == k + 1) {
          hr -= mur;
          hi = -mui;
        }
        double a_r = ar[j], a_i = ai[j];
        if (sw) {
          const double tr = a_r, ti = a_i;
          a_r = hr;
          a_i = hi;
          hr = tr;
          hi = ti;
        }
        if (j == k) {
          ur[j] = pr;
          ui[j] = pim;
        } else {
          ur[j] = a_r;
          ui[j] = a_i;
          ar[j] = hr - (lr * a_r - li * a_i);   // new active row
          ai[j] = hi - (lr * a_i + li * a_r);
        }
      }
#pragma unroll
      for (int t = 0; t < kMaxT; ++t) hrow[t] = hnext[t];
      if (lane == 0) {
        piv[k] = sw ? 1 : 0;
        mre[k] = lr;
        mim[k] = li;
      }
      __syncwarp();
    }
    {
      double* ur = Ur + off(n - 1) - (n - 1);
      double* ui = Ui + off(n - 1) - (n - 1);
      if (lane == 0) {
        double r_ = ar[n - 1], i_ = ai[n - 1];
        if (r_ == 0.0 && i_ == 0.0) r_ = tiny;
        ur[n - 1] = r_;
        ui[n - 1] = i_;
      }
    }
    __syncwarp();
    // y = L^{-1} P x (sequential, lane 0), then U y = that (column-oriented)
    if (lane == 0) {
      for (int i = 0; i < n; ++i) {
        yre[i] = xre[i];
        yim[i] = xim[i];
      }
      for (int k = 0; k + 1 < n; ++k) {
        if (piv[k]) {
          const double tr = yre[k], ti = yim[k];
          yre[k] = yre[k + 1];
          yim[k] = yim[k + 1];
          yre[k + 1] = tr;
          yim[k + 1] = ti;
        }
        const double lr = mre[k], li = mim[k];
        yre[k + 1] -= lr * yre[k] - li * yim[k];
        yim[k + 1] -= lr * yim[k] + li * yre[k];
      }
    }
    __syncwarp();
    for (int i = n - 1; i >= 0; --i) {
      const double uir = Ur[off(i)], uii = Ui[off(i)];
      const double iden = rcp_nr(uir * uir + uii * uii);
      const double br = yre[i], bi = yim[i];
      const double tr = (br * uir + bi * uii) * iden, ti = (bi * uir - br * uii) * iden;
      __syncwarp();
      if (lane == 0) {
        yre[i] = tr;
        yim[i] = ti;
      }
      for (int j = lane; j < i; j += 32) {   // y[j] -= U(j, i) y[i]
        const double cr = Ur[off(j) + (i - j)], ci = Ui[off(j) + (i - j)];
        yre[j] -= cr * tr - ci * ti;
        yim[j] -= cr * ti + ci * tr;
      }
      __syncwarp();
    }
    // Rayleigh quotient: theta = x^H y (x has unit norm); mu += 1 / theta
    double tr_ = 0.0, ti_ = 0.0, yy = 0.0;
    for (int i = lane; i < n; i += 32) {
      tr_ += xre[i] * yre[i] + xim[i] * yim[i];
      ti_ += xre[i] * yim[i] - xim[i] * yre[i];
      yy += yre[i] * yre[i] + yim[i] * yim[i];
    }
    tr_ = warp_sum(tr_);
    ti_ = warp_sum(ti_);
    yy = warp_sum(yy);
    const double den = tr_ * tr_ + ti_ * ti_;
    double dr = 0.0, di = 0.0;
    if (den > 0.0 && isfinite(den)) {
      dr = tr_ / den;
      di = -ti_ / den;
    }
    const double mag = hypot(mur, mui);
    if (hypot(dr, di) < 1e-3 * fmax(mag, 1e-300)) {
      mur += dr;
      if (pair) mui += di;   // a real eigenvalue stays real
    }
    const double inv = (yy > 0.0 && isfinite(yy)) ? 1.0 / sqrt(yy) : 1.0;
    for (int i = lane; i < n; i += 32) {
      xre[i] = yre[i] * inv;
      xim[i] = yim[i] * inv;
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) {
    Yre[i + (int64_t)blockIdx.x * n] = xre[i];
    Yim[i + (int64_t)blockIdx.x * n] = xim[i];
  }
  if (lane == 0) {
    wr[e] = mur;
    wi[e] = pair ? mui : 0.0;
    if (pair && e + 1 < n) {
      wr[e + 1] = mur;
      wi[e + 1] = -mui;
    }
  }
}

__global__ void k_normalize_complex(int n, double* Yre, double* Yim) {
  __shared__ double red[32];
  __shared__ int argmax;
  __shared__ double amax;
  double* yr = Yre + (int64_t)blockIdx.x * n;
  double* yi = Yim + (int64_t)blockIdx.x * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  double loc = 0.0;
  for (int i = tid; i < n; i += bd) loc += yr[i] * yr[i] + yi[i] * yi[i];
  const double nrm = sqrt(block_sum(loc, red));
  if (tid == 0) {
    int am = 0;
    double best = -1.0;
    for (int i = 0; i < n; ++i) {
      const double a = yr[i] * yr[i] + yi[i] * yi[i];
      if (a > best * (1.0 + 1e-12)) {   // first index wins near-ties: deterministic
        best = a;
        am = i;
      }
    }
    argmax = am;
    amax = sqrt(best);
  }
  __syncthreads();
  const double pr = yr[argmax], pi = yi[argmax];
  // multiply by conj(p)/|p| / nrm
  const double sc = (amax > 0.0 && nrm > 0.0) ? 1.0 / (amax * nrm) : 1.0;
  const double cr = pr * sc, ci = -pi * sc;
  __syncthreads();
  for (int i = tid; i < n; i += bd) {
    const double a = yr[i], b = yi[i];
    yr[i] = a * cr - b * ci;
    yi[i] = a * ci + b * cr;
  }
}

// Canonical order of the eigen-triplets and the real 2x2-block layout.
// Heads are the eigenvalues with wi >= 0 (one per conjugate pair).  Sorted by
// |lambda| descending, then Im descending (stable).  Writes, per output column
// c: lam_re[c], lam_im[c] and the real-form eigenvector column WR[:, c].
__global__ void k_eig_layout(int n, const double* __restrict__ wr, const double* __restrict__ wi,
                             const int* __restrict__ heads, const int* __restrict__ nheads_ptr,
                             const double* __restrict__ Yre,
                             const double* __restrict__ Yim, double* __restrict__ WR,
                             double* __restrict__ lam_re, double* __restrict__ lam_im,
                             int* __restrict__ order_scratch, int32_t* info) {
  __shared__ int colstart[1024];
  __shared__ double mag[1024];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nheads = min(*nheads_ptr, 1024);
  int* ord = order_scratch;
  for (int h = tid; h < nheads; h += bd) {
    const int e = heads[h];
    mag[h] = hypot(wr[e], wi[e]);
  }
  __syncthreads();
  // stable rank sort: |lambda| descending, then Im descending, then head index
  for (int h = tid; h < nheads; h += bd) {
    const double mh = mag[h], ih = wi[heads[h]];
    int rank = 0;
    for (int g = 0; g < nheads; ++g) {
      const double mg = mag[g], ig = wi[heads[g]];
      rank += (mg > mh) || (mg == mh && (ig > ih || (ig == ih && g < h)));
    }
    ord[rank] = h;
  }
  __syncthreads();
  if (tid == 0) {
    int c = 0, pairs = 0, reals = 0;
    for (int h = 0; h < nheads; ++h) {
      colstart[h] = c;
      const int e = heads[ord[h]];
      const int width = (wi[e] > 0.0) ? 2 : 1;
      if (c + width > n) {            // inconsistent pairing: never write past column n-1
        raise_status(info, DMD_ENUMERIC, 4998);
        colstart[h] = -1;
        continue;
      }
      if (wi[e] > 0.0) {
        lam_re[c] = wr[e]; lam_im[c] = wi[e];
        lam_re[c + 1] = wr[e]; lam_im[c + 1] = -wi[e];
        c += 2;
        ++pairs;
      } else {
        lam_re[c] = wr[e]; lam_im[c] = 0.0;
        c += 1;
        ++reals;
      }
    }
    if (info) {
      info[1] = pairs;
      info[2] = reals;
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  for (int h = warp; h < nheads; h += nw) {
    const int src = ord[h];
    const int e = heads[src];
    const int c = colstart[h];
    if (c < 0) continue;
    const bool pair = wi[e] > 0.0;
    for (int i = lane; i < n; i += 32) {
      WR[i + (int64_t)c * n] = Yre[i + (int64_t)src * n];
      if (pair) WR[i + (int64_t)(c + 1) * n] = Yim[i + (int64_t)src * n];
    }
  }
}

// heads[] = indices e with wi[e] >= 0 (in index order).  One thread.
__global__ void k_collect_heads(int n, const double* wi, int* heads, int* nheads, int32_t* info) {
  if (threadIdx.x != 0) return;
  int h = 0, c = 0;
  for (int e = 0; e < n; ++e) {
    if (wi[e] > 0.0) {
      heads[h++] = e;
      c += 2;
    } else if (wi[e] == 0.0) {
      heads[h++] = e;
      c += 1;
    } else if (!(wi[e] < 0.0)) {
      raise_status(info, DMD_ENUMERIC, 4000 + e);   // NaN eigenvalue
    }
  }
  if (c != n) raise_status(info, DMD_ENUMERIC, 4999);
  *nheads = h;
}

// ---------------------------------------- symmetric tridiagonal eigenproblem

// From a symmetric matrix reduced by k_hessenberg: d = diag, e = subdiagonal.
__device__ int sturm_count(int n, const double* d, const double* e, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e[i - 1] * e[i - 1] * rcp_nr(q);   // |q| >= pivmin: normal
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Eigenvalue i (descending) of the symmetric tridiagonal (d, e) -- the
// diagonal and subdiagonal of A after k_sytrd -- by warp multisection: each
// round the 32 lanes evaluate Sturm counts at 32 interior points and the
// bracket shrinks 33-fold; then lane 0 runs inverse iteration (3 solves with
// partial pivoting) for the eigenvector.  One warp per eigenvalue, so the
// FP64 work spreads over all SMs.  scratch: 7 n doubles per eigenvalue.
__global__ void k_tridiag_eig_ms(int n, const double* __restrict__ A, int lda, double* __restrict__ ev,
                                 double* __restrict__ Y, double* __restrict__ scratch) {
  extern __shared__ double sde[];
  double* d = sde;
  double* e = sde + n;
  const int i = blockIdx.x;
  const int lane = threadIdx.x;
  for (int t = lane; t < n; t += 32) {
    d[t] = A[t + (int64_t)t * lda];
    e[t] = (t + 1 < n) ? A[(t + 1) + (int64_t)t * lda] : 0.0;
  }
  __syncwarp();
  double lo = INFINITY, hi = -INFINITY, tnorm = 0.0;
  for (int t = lane; t < n; t += 32) {
    const double off = (t > 0 ? fabs(e[t - 1]) : 0.0) + (t + 1 < n ? fabs(e[t]) : 0.0);
    lo = fmin(lo, d[t] - off);
    hi = fmax(hi, d[t] + off);
    tnorm = fmax(tnorm, fabs(d[t]) + off);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  }
  if (tnorm == 0.0) tnorm = 1.0;
  const double pivmin = DBL_MIN * 4.0 + kEps * kEps * tnorm;
  lo -= 2.0 * kEps * tnorm;
  hi += 2.0 * kEps * tnorm;
  const int k = n - 1 - i;   // ascending index
  for (int round = 0; round < 14; ++round) {
    if (hi - lo <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    const double step = (hi - lo) / 33.0;
    const double x = lo + step * (lane + 1);
    const int cnt = sturm_count(n, d, e, x, pivmin);
    const unsigned mask = __ballot_sync(0xffffffffu, cnt > k);
    const int j = mask ? (__ffs(mask) - 1) : 32;   // first point with more than k eigenvalues below
    const double nlo = (j == 0) ? lo : lo + step * j;
    const double nhi = (j == 32) ? hi : lo + step * (j + 1);
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  const double lam = 0.5 * (lo + hi);
  ev[i] = lam;
  double* u0 = scratch + (int64_t)i * 7 * n;
  double* u1 = u0 + n;
  double* u2 = u1 + n;
  double* ml = u2 + n;
  double* pv = ml + n;
  double* xv = pv + n;
  const double tiny = kEps * tnorm;
  double c0 = d[0] - lam, c1 = (n > 1) ? e[0] : 0.0, c2 = 0.0;
  for (int q = 0; q + 1 < n; ++q) {
    const double b0 = e[q], b1 = d[q + 1] - lam, b2 = (q + 2 < n) ? e[q + 1] : 0.0;
    double p0, p1, p2, o0, o1, o2;
    if (fabs(b0) > fabs(c0)) {
      pv[q] = 1.0;
      p0 = b0; p1 = b1; p2 = b2; o0 = c0; o1 = c1; o2 = c2;
    } else {
      pv[q] = 0.0;
      p0 = c0; p1 = c1; p2 = c2; o0 = b0; o1 = b1; o2 = b2;
    }
    if (p0 == 0.0) p0 = tiny;
    const double mult = o0 / p0;
    u0[q] = p0; u1[q] = p1; u2[q] = p2; ml[q] = mult;
    c0 = o1 - mult * p1;
    c1 = o2 - mult * p2;
    c2 = 0.0;
  }
  if (c0 == 0.0) c0 = tiny;
  u0[n - 1] = c0; u1[n - 1] = 0.0; u2[n - 1] = 0.0;
  for (int t = 0; t < n; ++t) xv[t] = 1.0;
  for (int it = 0; it < 3; ++it) {
    for (int q = 0; q + 1 < n; ++q) {
      if (pv[q] != 0.0) {
        const double tt = xv[q];
        xv[q] = xv[q + 1];
        xv[q + 1] = tt;
      }
      xv[q + 1] -= ml[q] * xv[q];
    }
    for (int t = n - 1; t >= 0; --t) {
      double sacc = xv[t];
      if (t + 1 < n) sacc -= u1[t] * xv[t + 1];
      if (t + 2 < n) sacc -= u2[t] * xv[t + 2];
      xv[t] = sacc / u0[t];
    }
    double nrm = 0.0;
    for (int t = 0; t < n; ++t) nrm += xv[t] * xv[t];
    nrm = sqrt(nrm);
    const double inv = (nrm > 0.0 && isfinite(nrm)) ? 1.0 / nrm : 1.0;
    for (int t = 0; t < n; ++t) xv[t] *= inv;
  }
  for (int t = 0; t < n; ++t) Y[t + (int64_t)i * n] = xv[t];
}

// Modified Gram-Schmidt inside clusters of (nearly) equal eigenvalues, in
// descending order; one CTA.  Eigenvectors of well separated eigenvalues are
// left untouched.
__global__ void k_cluster_mgs(int n, const double* __restrict__ ev, double* __restrict__ Y, double rel) {
  __shared__ double red[32];
  const int tid = threadIdx.x, bd = blockDim.x;
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(ev[i]));
  const double gap = rel * (scale > 0.0 ? scale : 1.0);
  int start = 0;
  for (int i = 1; i < n; ++i) {
    if (fabs(ev[i - 1] - ev[i]) > gap) {
      start = i;
      continue;
    }
    double* yi = Y + (int64_t)i * n;
    for (int j = start; j < i; ++j) {
      const double* yj = Y + (int64_t)j * n;
      double loc = 0.0;
      for (int t = tid; t < n; t += bd) loc += yj[t] * yi[t];
      const double s = block_sum(loc, red);
      for (int t = tid; t < n; t += bd) yi[t] -= s * yj[t];
      __syncthreads();
    }
    double loc = 0.0;
    for (int t = tid; t < n; t += bd) loc += yi[t] * yi[t];
    const double nrm = sqrt(block_sum(loc, red));
    for (int t = tid; t < n; t += bd) yi[t] /= nrm;
    __syncthreads();
  }
}

// ------------------------------------------------------ least squares

// min || A X - B ||_F for A (mr x nc, ld, mr >= nc) and nrhs right-hand sides
// B (mr x nrhs, ld ldb) by Householder QR; A and B are overwritten; X is
// nc x nrhs (ld ldx).  One CTA; shared memory: mr + nc + nrhs + 32 doubles.
__global__ void k_lstsq(int mr, int nc, double* A, int ld, int nrhs, double* B, int ldb, double* X, int ldx,
                        int32_t* info) {
  extern __shared__ double sm[];
  double* v = sm;
  double* w = sm + mr;              // nc - 1 trailing columns + nrhs right-hand sides
  double* red = sm + mr + nc + nrhs;
  const int tid = threadIdx.x, bd = blockDim.x;
  double rmax = 0.0;
  const int ncol = nc + nrhs;       // columns of [A | B]
  auto colp = [&](int j) -> double* { return j < nc ? A + (int64_t)j * ld : B + (int64_t)(j - nc) * ldb; };
  for (int k = 0; k < nc; ++k) {
    double* col = A + (int64_t)k * ld;
    double loc = 0.0;
    for (int i = k + 1 + tid; i < mr; i += bd) loc += col[i] * col[i];
    const double sig = block_sum(loc, red);
    const double alpha = col[k];
    double tau = 0.0, beta = alpha;
    if (sig != 0.0) {
      const double nrm = sqrt(alpha * alpha + sig);
      beta = alpha <= 0.0 ? nrm : -nrm;
      tau = (beta - alpha) / beta;
      const double sc = 1.0 / (alpha - beta);
      for (int i = k + tid; i < mr; i += bd) v[i] = (i == k) ? 1.0 : col[i] * sc;
    } else {
      for (int i = k + tid; i < mr; i += bd) v[i] = (i == k) ? 1.0 : 0.0;
    }
    __syncthreads();
    rmax = fmax(rmax, fabs(beta));
    if (tau != 0.0) {
      for (int j = k + 1 + tid; j < ncol; j += bd) {
        const double* cj = colp(j);
        double s = 0.0;
        for (int i = k; i < mr; ++i) s = fma(v[i], cj[i], s);
        w[j - 1] = s;   // j >= k + 1
      }
      __syncthreads();
      const int wcols = ncol - k - 1;
      const int hgt = mr - k;
      for (int q = tid; q < wcols * hgt; q += bd) {
        const int i = k + q % hgt, j = k + 1 + q / hgt;
        colp(j)[i] -= tau * v[i] * w[j - 1];
      }
      __syncthreads();
    }
    if (tid == 0) col[k] = beta;
    for (int i = k + 1 + tid; i < mr; i += bd) col[i] = 0.0;
    __syncthreads();
  }
  for (int c = tid; c < nrhs; c += bd) {
    const double* b = B + (int64_t)c * ldb;
    double* x = X + (int64_t)c * ldx;
    for (int i = nc - 1; i >= 0; --i) {
      double s = b[i];
      for (int j = i + 1; j < nc; ++j) s -= A[i + (int64_t)j * ld] * x[j];
      const double piv = A[i + (int64_t)i * ld];
      if (fabs(piv) <= 1e-14 * rmax || !isfinite(piv)) {
        raise_status(info, DMD_ENUMERIC, 5000 + i);
        x[i] = 0.0;
      } else {
        x[i] = s / piv;
      }
    }
  }
}

// ------------------------------------------- shared-memory resident variants
//
// The same algorithms with the matrix held in shared memory (leading dimension
// n | 1, odd, so that a warp reading a row touches distinct banks): the
// global-memory versions above stream every column through L2 with strided,
// uncoalesced accesses, which dominates their run time.  Loops are arranged
// warp-per-column / lane-per-row (contiguous in shared memory), with no
// integer division.  Used whenever the matrix fits (n up to ~160).

constexpr size_t kSmallSmemMax = 220 * 1024;

// sum_i x[i * sx] y[i] with four independent accumulators: an FP64 FMA has
// ~64 cycles of latency on GB300, so a single chain would serialise on it.
__device__ __forceinline__ double dot4(const double* x, int sx, const double* y, int m) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = 0;
  for (; i + 3 < m; i += 4) {
    s0 = fma(x[i * sx], y[i], s0);
    s1 = fma(x[(i + 1) * sx], y[i + 1], s1);
    s2 = fma(x[(i + 2) * sx], y[i + 2], s2);
    s3 = fma(x[(i + 3) * sx], y[i + 3], s3);
  }
  for (; i < m; ++i) s0 = fma(x[i * sx], y[i], s0);
  return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ void load_square(double* S, int ldw, const double* G, int ld, int rows, int cols) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = warp; b < cols; b += nw)
    for (int a = lane; a < rows; a += 32) S[a + b * ldw] = G[a + (int64_t)b * ld];
}
__device__ __forceinline__ void store_square(double* G, int ld, const double* S, int ldw, int rows, int cols) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = warp; b < cols; b += nw)
    for (int a = lane; a < rows; a += 32) G[a + (int64_t)b * ld] = S[a + b * ldw];
}

// Cholesky as k_cholesky_upper (same pivot / drop rule), matrix in shared memory.
__global__ void k_cholesky_smem(int n, double* G, int ld, double tau, int32_t* info, int tag,
                                const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ double sm[];
  const int ldw = n | 1;
  double* S = sm;
  double* r = S + n * ldw;      // row j of R, contiguous
  double* red = r + n;
  __shared__ double piv, ipiv;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  for (int b = warp; b < n; b += nw)
    for (int a = lane; a <= b; a += 32) S[a + b * ldw] = G[a + (int64_t)b * ld];
  double loc = 0.0;
  for (int j = tid; j < n; j += bd) loc = fmax(loc, G[j + (int64_t)j * ld]);
  const double dmax = block_max(loc, red);
  const double floor_ = tau * dmax;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = S[j + j * ldw];
      if (!isfinite(d) || !isfinite(dmax)) {
        raise_status(info, DMD_ENONFINITE, tag * 1000 + j);
        piv = -1.0;
      } else if (!(dmax > 0.0)) {
        raise_status(info, DMD_ENUMERIC, tag * 1000 + j);
        piv = -1.0;
      } else if (!(d > floor_)) {
        piv = 0.0;   // dropped direction
        if (info) atomicAdd(&info[5], 1);
      } else {
        ipiv = rsqrt_nr(d);   // one lane: FP64 square root and division are slow
        piv = d * ipiv;
      }
      if (piv >= 0.0) S[j + j * ldw] = piv;
      if (!(piv > 0.0)) ipiv = 0.0;
    }
    __syncthreads();
    const double p = piv;
    if (p < 0.0) return;
    const double ip = ipiv;
    for (int i = j + 1 + tid; i < n; i += bd) {
      const double v = p == 0.0 ? 0.0 : S[j + i * ldw] * ip;
      S[j + i * ldw] = v;
      r[i] = v;
    }
    __syncthreads();
    if (p == 0.0) continue;
    for (int b = j + 1 + warp; b < n; b += nw) {
      const double rb = r[b];
      double* col = S + b * ldw;
      for (int a = j + 1 + lane; a <= b; a += 32) col[a] = fma(-r[a], rb, col[a]);
    }
    __syncthreads();
  }
  for (int b = warp; b < n; b += nw)
    for (int a = lane; a < n; a += 32) G[a + (int64_t)b * ld] = (a <= b) ? S[a + b * ldw] : 0.0;
}

// Cholesky as k_cholesky_smem in FP32 (input and output FP64).  For Gram
// matrices that are already close to the identity (the second pass of
// CholeskyQR2), where FP32 rounding (~1e-7) is far below the accuracy the
// basis is stored with.
__global__ void k_cholesky_f32(int n, double* G, int ld, double tau, int32_t* info, int tag,
                               const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ float smf[];
  const int ldw = n | 1;
  float* S = smf;
  float* r = S + n * ldw;
  __shared__ double red[32];
  __shared__ float piv;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  for (int b = warp; b < n; b += nw)
    for (int a = lane; a <= b; a += 32) S[a + b * ldw] = (float)G[a + (int64_t)b * ld];
  double loc = 0.0;
  for (int j = tid; j < n; j += bd) loc = fmax(loc, G[j + (int64_t)j * ld]);
  const double dmax = block_max(loc, red);
  const float floor_ = (float)(tau * dmax);
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const float d = S[j + j * ldw];
      if (!isfinite(d) || !isfinite(dmax)) {
        raise_status(info, DMD_ENONFINITE, tag * 1000 + j);
        piv = -1.f;
      } else if (!(dmax > 0.0)) {
        raise_status(info, DMD_ENUMERIC, tag * 1000 + j);
        piv = -1.f;
      } else if (!(d > floor_)) {
        piv = 0.f;
        if (info) atomicAdd(&info[5], 1);
      } else {
        piv = sqrtf(d);
      }
      if (piv >= 0.f) S[j + j * ldw] = piv;
    }
    __syncthreads();
    const float p = piv;
    if (p < 0.f) return;
    const float ip = p == 0.f ? 0.f : 1.f / p;
    for (int i = j + 1 + tid; i < n; i += bd) {
      const float v = p == 0.f ? 0.f : S[j + i * ldw] * ip;
      S[j + i * ldw] = v;
      r[i] = v;
    }
    __syncthreads();
    if (p == 0.f) continue;
    for (int b = j + 1 + warp; b < n; b += nw) {
      const float rb = r[b];
      float* col = S + b * ldw;
      for (int a = j + 1 + lane; a <= b; a += 32) col[a] = fmaf(-r[a], rb, col[a]);
    }
    __syncthreads();
  }
  for (int b = warp; b < n; b += nw)
    for (int a = lane; a < n; a += 32) G[a + (int64_t)b * ld] = (a <= b) ? (double)S[a + b * ldw] : 0.0;
}

// T = R^{-1}, one CTA per column j, column-oriented back substitution:
// b = e_j; for i = j .. 0: t_i = b_i / r_ii, b[0..i) -= t_i R[0..i, i].  No
// reductions: each step is one scaled column update spread over the lanes of
// one warp, so the FP64 work of the n columns runs on n SMs at once.  All
// warps of the CTA stage R's columns 0..j (upper part, packed) in shared
// memory first.
__global__ void __launch_bounds__(128) k_tri_inv_col(int n, const double* __restrict__ R, int ldr,
                                                     double* __restrict__ T, int ldt,
                                                     const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ double sm[];
  const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double* Rp = sm;                        // column i at offset i (i + 1) / 2
  double* b = Rp + (j + 1) * (j + 2) / 2;  // j + 1
  double* inv = b + (j + 1);               // j + 1
  for (int i = warp; i <= j; i += nw) {
    const int off = i * (i + 1) / 2;
    for (int a = lane; a <= i; a += 32) Rp[off + a] = R[a + (int64_t)i * ldr];
  }
  __syncthreads();
  if (warp != 0) return;
  for (int i = lane; i <= j; i += 32) {
    const double d = Rp[i * (i + 1) / 2 + i];
    inv[i] = d == 0.0 ? 0.0 : 1.0 / d;
    b[i] = (i == j) ? 1.0 : 0.0;
  }
  __syncwarp();
  double* out = T + (int64_t)j * ldt;
  for (int i = j + 1 + lane; i < n; i += 32) out[i] = 0.0;
  if (inv[j] == 0.0) {   // dropped direction: zero column
    for (int i = lane; i <= j; i += 32) out[i] = 0.0;
    return;
  }
  for (int i = j; i >= 0; --i) {
    const double ti = b[i] * inv[i];
    const double* col = Rp + i * (i + 1) / 2;
    __syncwarp();
    if (lane == 0) b[i] = ti;
    for (int a = lane; a < i; a += 32) b[a] = fma(-ti, col[a], b[a]);
    __syncwarp();
  }
  for (int i = lane; i <= j; i += 32) out[i] = b[i];
}

// X[:, c] = alpha G^{-1} Bm[:, c] + beta X[:, c] for c < ncols, with the
// Cholesky factor R (upper, R^T R = G, ld ldr; a zero diagonal entry marks a
// dropped direction, whose component is set to zero) by forward substitution
// R^T y = b and back substitution R x = y.  Every CTA stages R packed by
// columns in shared memory; each warp solves one right-hand side, the lanes
// sharing the scaled-column update of each step (no reductions).
__global__ void __launch_bounds__(512) k_chol_solve_cols(int n, const double* __restrict__ R, int ldr,
                                                         const double* __restrict__ Bm, int ldb, int ncols,
                                                         double alpha, double beta, double* __restrict__ X,
                                                         int ldx, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ double sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double* Rp = sm;                               // column i at offset i (i + 1) / 2
  double* inv = Rp + (size_t)n * (n + 1) / 2;    // n
  double* bw = inv + n + warp * n;               // this warp's right-hand side
  for (int i = warp; i < n; i += nw) {
    const int off = i * (i + 1) / 2;
    for (int a = lane; a <= i; a += 32) Rp[off + a] = R[a + (int64_t)i * ldr];
  }
  for (int i = tid; i < n; i += blockDim.x) {
    const double d = R[i + (int64_t)i * ldr];
    inv[i] = d == 0.0 ? 0.0 : 1.0 / d;
  }
  __syncthreads();
  const int c = blockIdx.x * nw + warp;
  if (c >= ncols) return;
  for (int i = lane; i < n; i += 32) bw[i] = Bm[i + (int64_t)c * ldb];
  __syncwarp();
  // R^T y = b: y_j = b_j / r_jj, then b_i -= r_ji y_j for i > j
  for (int j = 0; j < n; ++j) {
    const double yj = bw[j] * inv[j];
    __syncwarp();
    if (lane == 0) bw[j] = yj;
    for (int i = j + 1 + lane; i < n; i += 32) bw[i] = fma(-Rp[i * (i + 1) / 2 + j], yj, bw[i]);
    __syncwarp();
  }
  // R x = y: x_j = y_j / r_jj, then y_i -= r_ij x_j for i < j
  for (int j = n - 1; j >= 0; --j) {
    const double xj = bw[j] * inv[j];
    const double* col = Rp + j * (j + 1) / 2;
    __syncwarp();
    if (lane == 0) bw[j] = xj;
    for (int i = lane; i < j; i += 32) bw[i] = fma(-col[i], xj, bw[i]);
    __syncwarp();
  }
  double* out = X + (int64_t)c * ldx;
  for (int i = lane; i < n; i += 32) out[i] = beta == 0.0 ? alpha * bw[i] : fma(alpha, bw[i], beta * out[i]);
}

// Householder reflector of x[0..m) (x[0] = alpha): v (v[0] = 1) into v[],
// returns tau and beta; x itself is not modified.  Block-wide.  The scalar
// square root and divisions are taken by one thread and broadcast: on GB300's
// FP64 pipe (~2 DFMA/clk per SM) a block-wide redundant evaluation costs more
// than the reflector's vector work.
__device__ __forceinline__ void house(const double* x, int m, double* v, double* red, double& tau, double& beta) {
  __shared__ double hs[3];
  const int tid = threadIdx.x, bd = blockDim.x;
  double loc = 0.0;
  for (int i = 1 + tid; i < m; i += bd) loc += x[i] * x[i];
  const double sig = block_sum(loc, red);
  if (tid == 0) {
    const double alpha = x[0];
    if (sig == 0.0) {
      hs[0] = 0.0;
      hs[1] = alpha;
      hs[2] = 0.0;
    } else {
      const double nrm = sqrt(alpha * alpha + sig);
      const double bt = alpha <= 0.0 ? nrm : -nrm;
      hs[0] = (bt - alpha) / bt;
      hs[1] = bt;
      hs[2] = 1.0 / (alpha - bt);
    }
  }
  __syncthreads();
  tau = hs[0];
  beta = hs[1];
  const double sc = hs[2];
  for (int i = tid; i < m; i += bd) v[i] = (i == 0) ? 1.0 : x[i] * sc;
  __syncthreads();
}

// Tridiagonalisation as k_sytrd (same reflector storage), A in shared memory.
__global__ void k_sytrd_smem(int n, double* A, int ld, double* tau) {
  extern __shared__ double sm[];
  const int ldw = n | 1;
  double* S = sm;
  double* v = S + n * ldw;
  double* w = v + n;
  double* red = w + n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  load_square(S, ldw, A, ld, n, n);
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = S + k * ldw + (k + 1);
    double t, beta;
    house(x, m, v, red, t, beta);
    if (t == 0.0) {
      if (tid == 0) tau[k] = 0.0;
      continue;
    }
    for (int i = 1 + tid; i < m; i += bd) x[i] = v[i];
    if (tid == 0) {
      x[0] = beta;
      S[k + (k + 1) * ldw] = beta;
      tau[k] = t;
    }
    double* A22 = S + (k + 1) * ldw + (k + 1);
    // p = t * A22 v: row j of the symmetric A22 (contiguous across lanes = rows)
    for (int j = tid; j < m; j += bd) {
      double s = 0.0;
      s = dot4(A22 + j, ldw, v, m);
      w[j] = t * s;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = tid; i < m; i += bd) pv += w[i] * v[i];
    pv = block_sum(pv, red);
    for (int i = tid; i < m; i += bd) w[i] -= 0.5 * t * pv * v[i];
    __syncthreads();
    for (int j = warp; j < m; j += nw) {
      const double vj = v[j], wj = w[j];
      double* col = A22 + j * ldw;
      for (int i = lane; i < m; i += 32) col[i] -= v[i] * wj + w[i] * vj;
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) tau[k] = 0.0;
  }
  __syncthreads();
  store_square(A, ld, S, ldw, n, n);
}

// Hessenberg reduction as k_hessenberg (same reflector storage), A in shared memory.
__global__ void k_hessenberg_smem(int n, double* A, int ld, double* tau) {
  extern __shared__ double sm[];
  const int ldw = n | 1;
  double* S = sm;
  double* v = S + n * ldw;
  double* w = v + n;
  double* red = w + n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  load_square(S, ldw, A, ld, n, n);
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = S + k * ldw + (k + 1);
    double t, beta;
    house(x, m, v, red, t, beta);
    if (t == 0.0) {
      if (tid == 0) tau[k] = 0.0;
      continue;
    }
    for (int i = 1 + tid; i < m; i += bd) x[i] = v[i];
    if (tid == 0) {
      x[0] = beta;
      tau[k] = t;
    }
    // left: w_j = v . A[k+1.., j] for columns j = k+1.. (one thread per
    // column: no FP64 reductions); then A -= t v w^T
    for (int j = k + 1 + tid; j < n; j += bd) {
      const double* col = S + j * ldw + (k + 1);
      double s = 0.0;
      s = dot4(col, 1, v, m);
      w[j] = s;
    }
    __syncthreads();
    for (int j = k + 1 + warp; j < n; j += nw) {
      const double tw = t * w[j];
      double* col = S + j * ldw + (k + 1);
      for (int i = lane; i < m; i += 32) col[i] = fma(-v[i], tw, col[i]);
    }
    __syncthreads();
    // right: w_i = A[i, k+1..] . v for all rows i; then A -= t w v^T
    for (int i = tid; i < n; i += bd) {
      const double* row = S + (k + 1) * ldw + i;
      double s = 0.0;
      s = dot4(row, ldw, v, m);
      w[i] = s;
    }
    __syncthreads();
    for (int jj = warp; jj < m; jj += nw) {
      const double tv = t * v[jj];
      double* col = S + (k + 1 + jj) * ldw;
      for (int i = lane; i < n; i += 32) col[i] = fma(-w[i], tv, col[i]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) tau[k] = 0.0;
  }
  __syncthreads();
  store_square(A, ld, S, ldw, n, n);
}

// Least squares as k_lstsq, [A | B] in shared memory (mr x (nc + nrhs)).
__global__ void k_lstsq_smem(int mr, int nc, double* A, int ld, int nrhs, double* B, int ldb, double* X, int ldx,
                             int32_t* info) {
  extern __shared__ double sm[];
  const int ldw = mr | 1;
  const int ncol = nc + nrhs;
  double* S = sm;
  double* v = S + ncol * ldw;
  double* w = v + mr;
  double* red = w + ncol;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  load_square(S, ldw, A, ld, mr, nc);
  load_square(S + nc * ldw, ldw, B, ldb, mr, nrhs);
  __syncthreads();
  double rmax = 0.0;
  for (int k = 0; k < nc; ++k) {
    double* col = S + k * ldw;
    const int hgt = mr - k;
    double t, beta;
    house(col + k, hgt, v + k, red, t, beta);
    rmax = fmax(rmax, fabs(beta));
    if (t != 0.0) {
      for (int j = k + 1 + tid; j < ncol; j += bd) {   // one thread per column
        const double* cj = S + j * ldw;
        double s = 0.0;
        s = dot4(cj + k, 1, v + k, mr - k);
        w[j] = s;
      }
      __syncthreads();
      for (int j = k + 1 + warp; j < ncol; j += nw) {
        const double tw = t * w[j];
        double* cj = S + j * ldw;
        for (int i = k + lane; i < mr; i += 32) cj[i] = fma(-v[i], tw, cj[i]);
      }
    }
    __syncthreads();
    if (tid == 0) col[k] = beta;
    for (int i = k + 1 + tid; i < mr; i += bd) col[i] = 0.0;
    __syncthreads();
  }
  // back substitution, one warp per right-hand side (solution in shared memory)
  double* xsm = red + 32;
  for (int c = warp; c < nrhs; c += nw) {
    const double* b = S + (nc + c) * ldw;
    double* x = xsm + c * nc;
    for (int i = nc - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1 + lane; j < nc; j += 32) s = fma(S[i + j * ldw], x[j], s);
      s = b[i] - warp_sum(s);
      const double piv = S[i + i * ldw];
      if (lane == 0) {
        if (fabs(piv) <= 1e-14 * rmax || !isfinite(piv)) {
          raise_status(info, DMD_ENUMERIC, 5000 + i);
          x[i] = 0.0;
        } else {
          x[i] = s / piv;
        }
      }
      __syncwarp();
    }
    for (int i = lane; i < nc; i += 32) X[(int64_t)c * ldx + i] = x[i];
  }
}

}  // namespace

// ------------------------------------------------------------ launchers

dmd_status dgemm_gated(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B,
                       int ldb, bool tb, double beta, double* C, int ldc, const int32_t* skip, cudaStream_t st) {
  if (M <= 0 || N <= 0) return DMD_OK;
  dim3 grid((unsigned)ceil_div(M, 16), (unsigned)ceil_div(N, 16));
  k_dgemm<<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C, ldc, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status dgemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B,
                 int ldb, bool tb, double beta, double* C, int ldc, cudaStream_t st) {
  return dgemm_gated(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, nullptr, st);
}

// Shared-memory bytes of an n x n FP64 matrix with leading dimension n | 1
// plus `extra` doubles.
static size_t square_smem(int rows, int cols, size_t extra) {
  return ((size_t)(rows | 1) * cols + extra) * sizeof(double);
}

bool householder_cluster_fits(int n);
bool cholesky_cluster_fits(int n);
dmd_status cholesky_cluster(int n, double* G, int ld, double tau, int32_t* info, int tag, bool fp32,
                            const int32_t* skip, cudaStream_t st);
dmd_status hessenberg_cluster(int n, double* A, int ld, double* tau, cudaStream_t st);
dmd_status sytrd_cluster(int n, double* A, int ld, double* tau, cudaStream_t st);

static dmd_status set_smem(const void* fn, size_t bytes) {
  DMD_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return DMD_OK;
}

dmd_status cholesky_upper_gated(int n, double* G, int ld, double tau, int32_t* info, int tag, const int32_t* skip,
                                cudaStream_t st) {
  if (cholesky_cluster_fits(n)) return cholesky_cluster(n, G, ld, tau, info, tag, false, skip, st);
  const size_t smem = square_smem(n, n, (size_t)n + 32);
  if (smem <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_cholesky_smem, smem));
    k_cholesky_smem<<<1, 512, smem, st>>>(n, G, ld, tau, info, tag, skip);
  } else {
    k_cholesky_upper<<<1, 1024, 0, st>>>(n, G, ld, tau, info, tag, skip);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status cholesky_upper(int n, double* G, int ld, double tau, int32_t* info, int tag, cudaStream_t st) {
  return cholesky_upper_gated(n, G, ld, tau, info, tag, nullptr, st);
}

dmd_status tri_inv_upper_gated(int n, const double* R, int ldr, double* T, int ldt, const int32_t* skip,
                               cudaStream_t st) {
  const size_t smem = ((size_t)n * (n + 1) / 2 + 2 * (size_t)n) * sizeof(double);
  if (smem <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_tri_inv_col, smem));
    k_tri_inv_col<<<(unsigned)n, 128, smem, st>>>(n, R, ldr, T, ldt, skip);
  } else {
    k_tri_inv_upper<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(n, R, ldr, T, ldt, skip);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status chol_solve_gated(int n, const double* R, int ldr, const double* Bm, int ldb, int ncols, double alpha,
                            double beta, double* X, int ldx, const int32_t* skip, cudaStream_t st) {
  const int warps = 16;
  const size_t smem = ((size_t)n * (n + 1) / 2 + (size_t)n * (1 + warps)) * sizeof(double);
  DMD_REQUIRE(smem <= kSmallSmemMax, "chol_solve: n = %d too large for shared memory", n);
  DMD_TRY(set_smem((const void*)k_chol_solve_cols, smem));
  k_chol_solve_cols<<<(unsigned)ceil_div(ncols, warps), 32 * warps, smem, st>>>(n, R, ldr, Bm, ldb, ncols, alpha,
                                                                                beta, X, ldx, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status tri_inv_upper(int n, const double* R, int ldr, double* T, int ldt, cudaStream_t st) {
  return tri_inv_upper_gated(n, R, ldr, T, ldt, nullptr, st);
}

// FP32 factor of a near-identity Gram: one CTA while the FP32 matrix fits in
// its shared memory (measured faster than the 8-CTA cluster at n = 160: 190
// against 234 us, the FP32 updates being cheap next to the cluster
// barriers), the cluster beyond.
dmd_status cholesky_upper_f32_gated(int n, double* G, int ld, double tau, int32_t* info, int tag,
                                    const int32_t* skip, cudaStream_t st) {
  const size_t smem = ((size_t)(n | 1) * n + n) * sizeof(float);
  if (smem <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_cholesky_f32, smem));
    k_cholesky_f32<<<1, 512, smem, st>>>(n, G, ld, tau, info, tag, skip);
    DMD_LAUNCH_CHECK();
    return DMD_OK;
  }
  if (cholesky_cluster_fits(n)) return cholesky_cluster(n, G, ld, tau, info, tag, true, skip, st);
  return cholesky_upper_gated(n, G, ld, tau, info, tag, skip, st);
}

dmd_status cholesky_upper_f32(int n, double* G, int ld, double tau, int32_t* info, int tag, cudaStream_t st) {
  return cholesky_upper_f32_gated(n, G, ld, tau, info, tag, nullptr, st);
}

dmd_status hessenberg(int n, double* A, int ld, double* tau, cudaStream_t st) {
  if (householder_cluster_fits(n)) return hessenberg_cluster(n, A, ld, tau, st);
  const size_t smem_s = square_smem(n, n, 2 * (size_t)n + 32);
  if (smem_s <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_hessenberg_smem, smem_s));
    k_hessenberg_smem<<<1, 512, smem_s, st>>>(n, A, ld, tau);
  } else {
    const size_t smem = (2 * (size_t)n + 32) * sizeof(double);
    k_hessenberg<<<1, 1024, smem, st>>>(n, A, ld, tau);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status apply_q(int n, const double* A, int lda, const double* tau, double* Y, int ldy, int nvec,
                   cudaStream_t st) {
  if (nvec <= 0) return DMD_OK;
  k_apply_q<<<(unsigned)nvec, 128, 0, st>>>(n, A, lda, tau, Y, ldy);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

size_t hqr_smem_bytes(int n) {
  return (size_t)n * (n | 1) * sizeof(float) +
         (size_t)(2 * kMsBulges * kMsLd + 4 * kMsBulges + 2 * kMsBulges + kMsWarps + 1) * sizeof(float) + 16;
}
bool hqr_fits_smem(int n) { return hqr_smem_bytes(n) <= 200 * 1024; }

// FP32 Francis QR for the eigenvalue estimates (refined in FP64 by hess_eigvecs):
// multishift chains on one CTA when the matrix fits in shared memory.
dmd_status hqr(int n, const double* H, int ldh, double* wr, double* wi, double* scratch, int32_t* info,
               cudaStream_t st) {
  if (hqr_fits_smem(n)) {
    const size_t smem = hqr_smem_bytes(n);
    if (smem > 48 * 1024)
      DMD_CUDA_TRY(cudaFuncSetAttribute(k_hqr_ms, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_hqr_ms<<<1, 32 * kMsWarps, smem, st>>>(n, H, ldh, wr, wi, info);
  } else {
    k_hqr<float, false><<<1, 32, 0, st>>>(n, H, ldh, wr, wi, reinterpret_cast<float*>(scratch), info);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status collect_heads(int n, const double* wi, int* heads, int* nheads, int32_t* info, cudaStream_t st) {
  k_collect_heads<<<1, 32, 0, st>>>(n, wi, heads, nheads, info);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

// Launched with the maximum possible number of heads (n); CTAs beyond the
// actual count exit (the head list is padded with -1 by the caller).
dmd_status hess_eigvecs(int n, const double* H, int ldh, const double* wr, const double* wi,
                        const int* heads, int nheads_max, double* Yre, double* Yim, double* work,
                        const double* hnorm, cudaStream_t st) {
  const size_t smem_w = ((size_t)n * (n + 1) + 8 * (size_t)n) * sizeof(double) + (size_t)n * sizeof(int) + 16;
  if (n <= 160 && smem_w <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_hess_rqi_w, smem_w));
    k_hess_rqi_w<<<(unsigned)nheads_max, 32, smem_w, st>>>(n, H, ldh, const_cast<double*>(wr),
                                                            const_cast<double*>(wi), heads, Yre, Yim, hnorm);
    DMD_LAUNCH_CHECK();
    return DMD_OK;
  }
  const size_t smem = (6 * (size_t)n) * sizeof(double) + (size_t)n * sizeof(int) + 16;
  k_hess_rqi<<<(unsigned)nheads_max, 256, smem, st>>>(n, H, ldh, const_cast<double*>(wr), const_cast<double*>(wi),
                                                       heads, Yre, Yim, work, hnorm);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status normalize_complex(int n, double* Yre, double* Yim, int ncols, cudaStream_t st) {
  if (ncols <= 0) return DMD_OK;
  k_normalize_complex<<<(unsigned)ncols, 128, 0, st>>>(n, Yre, Yim);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status eig_layout(int n, const double* wr, const double* wi, const int* heads, const int* nheads,
                      const double* Yre, const double* Yim, double* WR, double* lam_re, double* lam_im,
                      int* order_scratch, int32_t* info, cudaStream_t st) {
  k_eig_layout<<<1, 256, 0, st>>>(n, wr, wi, heads, nheads, Yre, Yim, WR, lam_re, lam_im, order_scratch,
                                  info);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status sytrd(int n, double* A, int ld, double* tau, cudaStream_t st) {
  if (householder_cluster_fits(n)) return sytrd_cluster(n, A, ld, tau, st);
  const size_t smem_s = square_smem(n, n, 2 * (size_t)n + 32);
  if (smem_s <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_sytrd_smem, smem_s));
    k_sytrd_smem<<<1, 512, smem_s, st>>>(n, A, ld, tau);
  } else {
    const size_t smem = (3 * (size_t)n + 32) * sizeof(double);
    k_sytrd<<<1, 1024, smem, st>>>(n, A, ld, tau);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status tridiag_eig(int n, const double* A, int lda, double* ev, double* Y, double* scratch,
                       cudaStream_t st) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  k_tridiag_eig_ms<<<(unsigned)n, 32, smem, st>>>(n, A, lda, ev, Y, scratch);
  DMD_LAUNCH_CHECK();
  k_cluster_mgs<<<1, 256, 0, st>>>(n, ev, Y, 1e-11);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status lstsq(int mr, int nc, double* A, int ld, int nrhs, double* B, int ldb, double* X, int ldx,
                 int32_t* info, cudaStream_t st) {
  const size_t smem_s = square_smem(mr, nc + nrhs, (size_t)mr + nc + nrhs + 32 + (size_t)nrhs * nc);
  if (smem_s <= kSmallSmemMax) {
    DMD_TRY(set_smem((const void*)k_lstsq_smem, smem_s));
    k_lstsq_smem<<<1, 512, smem_s, st>>>(mr, nc, A, ld, nrhs, B, ldb, X, ldx, info);
  } else {
    const size_t smem = ((size_t)mr + nc + nrhs + 32) * sizeof(double);
    k_lstsq<<<1, 256, smem, st>>>(mr, nc, A, ld, nrhs, B, ldb, X, ldx, info);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

}  // namespace dmd
