// C ABI of libdmd: argument checks, workspace carving and the orchestration
// of the fit, prediction and adjoint on the caller's stream.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "optdmd.cuh"

namespace dmd {

// ---- host error string and launch counter -----------------------------------
static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

// ---- kernels implemented in the other translation units ----------------------
dmd_status launch_sketch(int m, int l, uint64_t seed, double* Om, cudaStream_t st);
dmd_status launch_philox_blocks(int64_t count, uint32_t sid, uint64_t key, uint32_t* out, cudaStream_t st);
int tn_splits(int64_t n, int Ka, int N);
size_t tn_partial_doubles(int64_t n, int Ka, int N);
dmd_status f32_gemm_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const float* B32, float* C,
                       int64_t ldc, cudaStream_t st, const int32_t* skip);
dmd_status f32_gemm_tn(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
                       double* C, double* part, cudaStream_t st, const int32_t* skip);
dmd_status f64_to_f32(int64_t count, const double* in, float* out, cudaStream_t st, const int32_t* skip);
size_t umma_nn_workspace_bytes(int64_t n, int Kd, int N);
dmd_status umma_gemm_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, float* C,
                        int64_t ldc, void* ws, cudaStream_t st, int spare_sms, const int32_t* skip);
size_t umma_tn_workspace_bytes(int64_t n, int Ka, int N);
dmd_status umma_gemm_tn(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
                        double* C, int nsplit, void* ws, cudaStream_t st);
dmd_status launch_edit_modes(int r, int q, const double* in, double* out, double thr, const double* low,
                             const double* high, double dt, cudaStream_t st);
dmd_status umma_tune_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, float* C, int64_t ldc,
                        void* ws, cudaStream_t st, int32_t* chosen);
dmd_status umma_gemm_tn_flush(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
                              double* C, int nsplit, int flush, void* ws, cudaStream_t st, const int32_t* skip);
dmd_status dgemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B, int ldb,
                 bool tb, double beta, double* C, int ldc, cudaStream_t st);
dmd_status cholesky_upper(int n, double* G, int ld, double tau, int32_t* info, int tag, cudaStream_t st);
dmd_status cholesky_upper_f32(int n, double* G, int ld, double tau, int32_t* info, int tag, cudaStream_t st);
dmd_status tri_inv_upper(int n, const double* R, int ldr, double* T, int ldt, cudaStream_t st);
dmd_status hessenberg(int n, double* A, int ld, double* tau, cudaStream_t st);
dmd_status sytrd(int n, double* A, int ld, double* tau, cudaStream_t st);
dmd_status apply_q(int n, const double* A, int lda, const double* tau, double* Y, int ldy, int nvec,
                   cudaStream_t st);
dmd_status hqr(int n, const double* H, int ldh, double* wr, double* wi, double* scratch, int32_t* info,
               cudaStream_t st);
dmd_status collect_heads(int n, const double* wi, int* heads, int* nheads, int32_t* info, cudaStream_t st);
dmd_status hess_eigvecs(int n, const double* H, int ldh, const double* wr, const double* wi, const int* heads,
                        int nheads_max, double* Yre, double* Yim, double* work, const double* hnorm,
                        cudaStream_t st);
dmd_status normalize_complex(int n, double* Yre, double* Yim, int ncols, cudaStream_t st);
dmd_status eig_layout(int n, const double* wr, const double* wi, const int* heads, const int* nheads,
                      const double* Yre, const double* Yim, double* WR, double* lam_re, double* lam_im,
                      int* order_scratch, int32_t* info, cudaStream_t st);
dmd_status tridiag_eig(int n, const double* A, int lda, double* ev, double* Y, double* scratch, cudaStream_t st);
dmd_status lstsq(int mr, int nc, double* A, int ld, int nrhs, double* B, int ldb, double* X, int ldx,
                 int32_t* info, cudaStream_t st);
dmd_status launch_coefficients(int r, int K, const double* modal, const int32_t* ks, double* C, cudaStream_t st);
dmd_status launch_upsample_coeffs(int r, int T, const double* modal, double thr, double dt, const double* P,
                                  double* C, cudaStream_t st);
dmd_status launch_advect(int dim, int N, const float* rho, float* out, const float* u, float dt, cudaStream_t st);
dmd_status launch_iota(int32_t* out, int count, int start, cudaStream_t st);
dmd_status chol_solve_gated(int n, const double* R, int ldr, const double* Bm, int ldb, int ncols, double alpha,
                            double beta, double* X, int ldx, const int32_t* skip, cudaStream_t st);
dmd_status launch_rollout(int r, int q, int steps, const double* modal, const float* u, double* Xi,
                          cudaStream_t st);
dmd_status launch_gather_cols(int r, int K, const double* Xi, const int32_t* ks, int steps, double* C,
                              int32_t* info, cudaStream_t st);
dmd_status launch_chain_closed(int r, int K, const double* modal, const int32_t* ks, const double* dC,
                               double* dmodal, cudaStream_t st);
dmd_status launch_rollout_adjoint(int r, int q, int steps, int K, const int32_t* ks, const double* modal,
                                  const float* u, const double* Xi, const double* dC, double* dXi, double* Mu,
                                  double* dmodal, float* du, cudaStream_t st);
int loss_blocks();
dmd_status launch_loss_chunk(int64_t n, int nf, float* F, int64_t ldf, const float* tgt, const double* w,
                             bool grad, float delta, double* partial, double* loss, bool accumulate, cudaStream_t st);
dmd_status launch_sum_partials(int count, const double* partial, double* out, bool accumulate, cudaStream_t st);
int umma_loss_parts(int64_t n);
dmd_status umma_loss_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, const float* tgt,
                        const double* w, float delta, double* part, int* parts, void* ws, cudaStream_t st);
bool umma_loss_grad_supported(int r);
size_t umma_loss_grad_workspace_bytes(int64_t n, int r, int K);
dmd_status umma_loss_grad(int64_t n, int r, int K, const float* Phi, int64_t ldPhi, const double* C,
                          const float* tgt, const double* w, float delta, double* dC, double* loss_part, int* parts,
                          void* ws, cudaStream_t st);
dmd_status fit_glue_sigma(int l, int r, const double* ev, double* sigma, double* inv_sq, int32_t* info,
                          cudaStream_t st);
dmd_status fit_glue_scale_cols(int rows, int cols, double* A, int lda, const double* s, cudaStream_t st);
dmd_status fit_glue_check_finite(int64_t count, const double* A, int32_t* info, int tag, cudaStream_t st);
dmd_status fit_glue_maxabs(int64_t count, const double* A, double* out, cudaStream_t st);
dmd_status fit_glue_copy(int64_t count, const double* src, double* dst, cudaStream_t st);
dmd_status fit_glue_fill_int(int64_t count, int* dst, int v, cudaStream_t st);
dmd_status fit_glue_gate(int32_t* info, int32_t* gate, int mode, int spare, cudaStream_t st);
dmd_status fit_glue_shift_diag(int n, double* G, int ld, double rel, const int32_t* skip, cudaStream_t st);
dmd_status dgemm_gated(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B,
                       int ldb, bool tb, double beta, double* C, int ldc, const int32_t* skip, cudaStream_t st);
dmd_status cholesky_upper_gated(int n, double* G, int ld, double tau, int32_t* info, int tag, const int32_t* skip,
                                cudaStream_t st);
dmd_status tri_inv_upper_gated(int n, const double* R, int ldr, double* T, int ldt, const int32_t* skip,
                               cudaStream_t st);
dmd_status cholesky_upper_f32_gated(int n, double* G, int ld, double tau, int32_t* info, int tag,
                                    const int32_t* skip, cudaStream_t st);
dmd_status fit_glue_stack(int l, int q, int m, const double* P, const float* Ups, double* Om, cudaStream_t st);
dmd_status fit_glue_sigma_range(int L, int p, const double* ev, double* sigma_or_null, double* inv_sq, int32_t* info,
                                int tag, cudaStream_t st);

namespace {

// ---------------------------------------------------------- side streams
//
// A few small solves of the fit are independent of the tall pass running at
// the same time (the amplitudes' least squares beside the modes pass): they
// are forked onto a side stream of the caller's stream and joined back with
// events, so the caller's stream still orders all of the call's work and a
// capture of it records the fork and the join.  Side streams and events are
// created on first use, per (device, caller stream); a call made while a
// stream capture is in progress must therefore not be the first on its
// stream.  When the table is full the work simply stays on the caller's
// stream.
struct Side {
  int dev = -1;
  cudaStream_t origin = nullptr, side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxSides = 128;
Side g_sides[kMaxSides];
std::mutex g_side_mu;

const Side* side_of(cudaStream_t origin) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_side_mu);
  for (int i = 0; i < kMaxSides; ++i) {
    Side& s = g_sides[i];
    if (s.side != nullptr && s.dev == dev && s.origin == origin) return &s;
    if (s.side == nullptr) {
      Side t;
      t.dev = dev;
      t.origin = origin;
      if (cudaStreamCreateWithFlags(&t.side, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      if (cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&t.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(t.side);
        return nullptr;
      }
      s = t;
      return &s;
    }
  }
  return nullptr;
}

// ---------------------------------------------------------- precision dispatch

struct Tall {
  int prec;
  // scratch for the small FP64 operand rounded to FP32 / split (NN), and the
  // split partials (TN); carved once per call site.
  // The tensor-core NN kernels keep up to 256 inner-dimension columns
  // resident; a longer inner dimension (more than 256 snapshots) takes the
  // FP32 CUDA-core product in either form.
  bool nn_tensor(int Kd) const { return prec == DMD_MIXED_BF16X3 && Kd <= 256; }
  size_t nn_bytes(int64_t n, int Kd, int N) const {
    if (nn_tensor(Kd)) return umma_nn_workspace_bytes(n, Kd, N);
    return (size_t)Kd * N * sizeof(float) + 256;
  }
  size_t tn_bytes(int64_t n, int Ka, int N) const {
    if (prec == DMD_MIXED_BF16X3) return umma_tn_workspace_bytes(n, Ka, N);
    return tn_partial_doubles(n, Ka, N) * sizeof(double) + 256;
  }
  // skip: optional device flag; nonzero makes every launch of the product
  // return at once (work a device-side decision made unnecessary)
  dmd_status nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, float* C, int64_t ldc,
                void* ws, cudaStream_t st, int spare_sms = 0, const int32_t* skip = nullptr) const {
    if (nn_tensor(Kd)) return umma_gemm_nn(n, Kd, N, A, lda, B, C, ldc, ws, st, spare_sms, skip);
    float* B32 = reinterpret_cast<float*>(ws);
    DMD_TRY(f64_to_f32((int64_t)Kd * N, B, B32, st, skip));
    return f32_gemm_nn(n, Kd, N, A, lda, B32, C, ldc, st, skip);
  }
  // The snapshot Gram W = S^T S on the CUDA cores in both forms: the first
  // CholeskyQR Gram of every sketch is derived from it, and a random sketch
  // of the leading subspace can be conditioned far worse than the snapshots
  // (cond(Y)^2 up to ~1e10 was seen for l = r); FP32 products summed in
  // 32-row tiles and carried in FP64 resolve that, the tensor-core
  // accumulation does not (measured: ~2e-8 of the largest eigenvalue).
  size_t tn_accurate_bytes(int64_t n, int Ka, int N) const {
    return tn_partial_doubles(n, Ka, N) * sizeof(double) + 256;
  }
  dmd_status tn_accurate(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
                         double* C, void* ws, cudaStream_t st, const int32_t* skip = nullptr) const {
    return f32_gemm_tn(n, Ka, N, A, lda, B, ldb, C, reinterpret_cast<double*>(ws), st, skip);
  }
  dmd_status tn(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb, double* C,
                void* ws, cudaStream_t st, const int32_t* skip = nullptr) const {
    // BF16x3 (hi/lo split, 3 products), TMEM flushed to FP64 in segments
    // sized by the row count (16 .. 256 k-steps).  The reductions that see the snapshots' full dynamic range
    // (the snapshot Gram) run on the CUDA cores instead (tn_accurate).
    if (prec == DMD_MIXED_BF16X3) return umma_gemm_tn_flush(n, Ka, N, A, lda, B, ldb, C, 2, 0, ws, st, skip);
    return f32_gemm_tn(n, Ka, N, A, lda, B, ldb, C, reinterpret_cast<double*>(ws), st, skip);
  }
};

bool valid_precision(int p) { return p == DMD_FP32 || p == DMD_MIXED_BF16X3; }

// ---------------------------------------------------------------- fit layout

struct FitBufs {
  int64_t n, ldY;
  int m, r, l, q, lo;   // lo = rows of the "input" sketch (m); control stacks q extra rows
  double *Om, *G, *T1, *T2, *Zp, *Z, *Gz, *Tz, *P, *Pp, *Hb, *tauB, *evB, *YB, *trid, *Vs, *Tmp, *At, *Ah,
      *tauA, *Hq, *wr, *wi, *Yre, *Yim, *invit, *WR, *MR, *LS, *rhs, *hnorm, *invsq;
  float* Q1;
  int *heads, *nheads, *order;
  double* G0;      // the first Gram, kept for the shifted fallback
  int32_t* gate;   // [2] fallback gate (k_gate)
  // DMD with control (q > 0): input-space SVD of [Q^T X; Ups] and its products
  double *W, *WB;   // snapshot Gram S^T S ((m+1) x (m+1)) and W_X B (m x l)
  int L, p;
  double *Omc, *Hc, *tauC, *evC, *YC, *tridC, *VS, *T1c, *T2c, *Tw, *invC, *rhsc, *solc;
  void* gemm_ws;
  size_t gemm_ws_bytes;
};

void carve_fit(Arena& a, const dmd_fit_desc& d, const Tall& tall, FitBufs& b) {
  b.n = d.n;
  b.m = d.m;
  b.r = d.r;
  b.q = d.q;
  b.l = std::min(d.r + std::max(d.oversample, 0), d.m);
  b.ldY = round_up(d.n, 32);
  const int m = b.m, l = b.l, r = b.r;
  const int64_t n = b.n;
  b.Om = a.take<double>((size_t)m * l);
  b.W = a.take<double>((size_t)(m + 1) * (m + 1));
  b.WB = a.take<double>((size_t)m * l);
  b.G = a.take<double>((size_t)l * l);
  b.T1 = a.take<double>((size_t)l * l);
  b.T2 = a.take<double>((size_t)l * l);
  b.Zp = a.take<double>((size_t)m * l);
  b.Z = a.take<double>((size_t)m * l);
  b.Gz = a.take<double>((size_t)l * l);
  b.Tz = a.take<double>((size_t)l * l);
  b.P = a.take<double>((size_t)l * (m + 1));
  b.Pp = a.take<double>((size_t)l * (m + 1));
  b.Hb = a.take<double>((size_t)l * l);
  b.tauB = a.take<double>(l);
  b.evB = a.take<double>(l);
  b.YB = a.take<double>((size_t)l * l);
  b.trid = a.take<double>((size_t)7 * l * l);
  b.Vs = a.take<double>((size_t)m * r);
  b.Tmp = a.take<double>((size_t)l * r);
  b.At = a.take<double>((size_t)r * r);
  b.Ah = a.take<double>((size_t)r * r);
  b.tauA = a.take<double>(r);
  b.Hq = a.take<double>((size_t)r * r);
  b.wr = a.take<double>(r);
  b.wi = a.take<double>(r);
  b.Yre = a.take<double>((size_t)r * r);
  b.Yim = a.take<double>((size_t)r * r);
  b.invit = a.take<double>((size_t)2 * r * r * r);
  b.WR = a.take<double>((size_t)r * r);
  b.MR = a.take<double>((size_t)m * r);
  b.LS = a.take<double>((size_t)l * r);
  b.rhs = a.take<double>(l);
  b.hnorm = a.take<double>(1);
  b.invsq = a.take<double>(l);
  b.heads = a.take<int>(r);
  b.nheads = a.take<int>(1);
  b.order = a.take<int>(r);
  b.G0 = a.take<double>((size_t)l * l);
  b.gate = a.take<int32_t>(4);
  b.Q1 = a.take<float>((size_t)b.ldY * l);
  b.L = l + d.q;
  b.p = std::min(d.r + d.q, std::min(b.L, m));
  if (d.q > 0) {
    const int L = b.L, pp = b.p, q = d.q;
    b.Omc = a.take<double>((size_t)L * m);
    b.Hc = a.take<double>((size_t)L * L);
    b.tauC = a.take<double>(L);
    b.evC = a.take<double>(L);
    b.YC = a.take<double>((size_t)L * L);
    b.tridC = a.take<double>((size_t)7 * L * L);
    b.VS = a.take<double>((size_t)m * pp);
    b.T1c = a.take<double>((size_t)l * pp);
    b.T2c = a.take<double>((size_t)pp * r);
    b.Tw = a.take<double>((size_t)pp * r);
    b.invC = a.take<double>(L);
    b.rhsc = a.take<double>((size_t)l * (q + 1));
    b.solc = a.take<double>((size_t)r * (q + 1));
  }
  size_t g = 0;
  g = std::max(g, tall.nn_bytes(n, m, l));
  g = std::max(g, tall.nn_bytes(n, l, l));
  g = std::max(g, tall.nn_bytes(n, m, r));
  g = std::max(g, tall.tn_bytes(n, l, l));
  g = std::max(g, tall.tn_bytes(n, m, l));
  g = std::max(g, tall.tn_bytes(n, l, m + 1));
  g = std::max(g, tall.tn_accurate_bytes(n, m + 1, m + 1));
  g = std::max(g, tall.tn_accurate_bytes(n, l, l));   // the shifted fallback's accurate Gram
  b.gemm_ws_bytes = g;
  b.gemm_ws = a.take<char>(g, 1024);
}

dmd_status validate_fit(const dmd_fit_desc* d) {
  DMD_REQUIRE(d != nullptr, "dmd_fit: desc is NULL");
  DMD_REQUIRE(d->n >= 1 && d->m >= 2, "dmd_fit: need n >= 1 and m >= 2 (got n=%lld m=%d)", (long long)d->n, d->m);
  DMD_REQUIRE(d->r >= 1 && d->r <= d->m && d->r <= d->n, "dmd_fit: need 1 <= r <= min(m, n) (r=%d)", d->r);
  DMD_REQUIRE(d->r <= 512, "dmd_fit: r > 512 is not supported");
  DMD_REQUIRE(d->oversample >= 0 && d->power_iters >= 0 && d->power_iters <= 16, "dmd_fit: bad oversample/power_iters");
  DMD_REQUIRE(d->ldS >= d->n && d->ldS % 4 == 0, "dmd_fit: ldS must be >= n and a multiple of 4");
  DMD_REQUIRE(d->ldPhi >= d->n && d->ldPhi % 4 == 0, "dmd_fit: ldPhi must be >= n and a multiple of 4");
  DMD_REQUIRE(d->q >= 0 && d->q <= 64, "dmd_fit: q must be in [0, 64]");
  DMD_REQUIRE(valid_precision(d->precision), "dmd_fit: unknown precision %d", d->precision);
  const int l = std::min(d->r + d->oversample, d->m);
  DMD_REQUIRE(l <= 1024, "dmd_fit: sketch width above 1024");
  return DMD_OK;
}

// Relative pivot floor of the Gram-based orthonormalisations: a direction
// whose squared residual is below tau * (largest squared column norm) is
// dropped.  The tall Grams are accurate to ~1e-6 relative (FP32 / split-bf16
// products summed in FP32 over short stretches, FP64 across), so 1e-10 keeps
// every direction the data resolve and drops the rounding-noise ones; the
// small FP64 Grams use 1e-13.
constexpr double kTauTall = 1e-10, kTauSmall = 1e-13;

// Shifted CholeskyQR3 fallback of orth_tall (every launch returns at once
// unless the first Cholesky factorisation dropped more directions than the
// l - r spare columns of the sketch: b.gate[1] is then 0).  The sketch Y = X Bs then holds directions below what the FP64
// first Gram resolves after the FP32 snapshot products (about 1e-5 sigma_1);
// instead of dropping them:
//   1. R1 = chol(G + s I), s = 1e-6 max_i G_ii: every pivot is at least s,
//      and Q1 = Y R1^{-1} has condition number at most ~1e3 (the weak
//      directions are damped, not lost);
//   2. R2 = chol(Q1^T Q1) with Q1^T Q1 taken by the FP32 CUDA-core reduction
//      with FP64 carries (accurate to ~1e-10 of its norm, enough for that
//      condition number), and the basis formed again from the snapshots,
//      Q2 = X (Bs R1^{-1} R2^{-1}), overwriting Q1;
//   3. the usual second pass on Q2: R3 = chol(Q2^T Q2), T2 = R3^{-1}.
// Consumers then use Q = Q2 T2 as after the plain pass.
dmd_status orth_tall_shifted(const Tall& tall, FitBufs& b, const float* X, int64_t ldX, const double* Bs,
                             int32_t* info, int tag, cudaStream_t st) {
  const int l = b.l, m = b.m;
  const int32_t* skip = b.gate + 1;
  DMD_TRY(fit_glue_shift_diag(l, b.G0, l, 1e-6, skip, st));
  DMD_TRY(cholesky_upper_gated(l, b.G0, l, 0.0, info, tag + 2, skip, st));
  DMD_TRY(tri_inv_upper_gated(l, b.G0, l, b.T1, l, skip, st));
  DMD_TRY(dgemm_gated(m, l, l, 1.0, Bs, m, false, b.T1, l, false, 0.0, b.WB, m, skip, st));    // Bs R1^{-1}
  DMD_TRY(tall.nn(b.n, m, l, X, ldX, b.WB, b.Q1, b.ldY, b.gemm_ws, st, 0, skip));
  DMD_TRY(tall.tn_accurate(b.n, l, l, b.Q1, b.ldY, b.Q1, b.ldY, b.G0, b.gemm_ws, st, skip));
  DMD_TRY(cholesky_upper_gated(l, b.G0, l, kTauSmall, info, tag + 3, skip, st));
  DMD_TRY(tri_inv_upper_gated(l, b.G0, l, b.T2, l, skip, st));
  DMD_TRY(dgemm_gated(l, l, l, 1.0, b.T1, l, false, b.T2, l, false, 0.0, b.G, l, skip, st));   // R1^{-1} R2^{-1}
  DMD_TRY(dgemm_gated(m, l, l, 1.0, Bs, m, false, b.G, l, false, 0.0, b.WB, m, skip, st));
  DMD_TRY(tall.nn(b.n, m, l, X, ldX, b.WB, b.Q1, b.ldY, b.gemm_ws, st, 0, skip));
  DMD_TRY(tall.tn(b.n, l, l, b.Q1, b.ldY, b.Q1, b.ldY, b.G0, b.gemm_ws, st, skip));
  DMD_TRY(cholesky_upper_f32_gated(l, b.G0, l, kTauTall, info, tag + 4, skip, st));
  DMD_TRY(tri_inv_upper_gated(l, b.G0, l, b.T2, l, skip, st));
  return DMD_OK;
}

// CholeskyQR2 of the tall sketch Y = X Bs (n x l, Bs = Omega or Z, m x l):
// the first Gram is formed in the small space as Bs^T (X^T X) Bs from the
// snapshot Gram W (one accurate pass over S per fit), so it carries FP64
// accuracy whatever the condition of Y.  Y itself is never stored: the first
// orthonormal factor is one tall product Q1 = Y R1^{-1} = X (Bs R1^{-1}).
// The second Gram Q1^T Q1 (of a well-conditioned matrix, close to I) is a
// tall reduction and its Cholesky factor is taken in FP32; the second factor
// is kept as T2 = R2^{-1} and folded into the consumers (Q = Q1 T2).
dmd_status orth_tall(const Tall& tall, FitBufs& b, const float* X, int64_t ldX, const double* Bs, int32_t* info,
                     int tag, cudaStream_t st) {
  const int l = b.l, m = b.m;
  DMD_TRY(dgemm(m, l, m, 1.0, b.W, m + 1, false, Bs, m, false, 0.0, b.WB, m, st));
  DMD_TRY(dgemm(l, l, m, 1.0, Bs, m, true, b.WB, m, false, 0.0, b.G, l, st));
  DMD_TRY(fit_glue_copy((int64_t)l * l, b.G, b.G0, st));
  DMD_TRY(fit_glue_gate(info, b.gate, 0, 0, st));
  DMD_TRY(cholesky_upper(l, b.G, l, kTauTall, info, tag, st));
  DMD_TRY(fit_glue_gate(info, b.gate, 1, l - b.r, st));
  DMD_TRY(tri_inv_upper(l, b.G, l, b.T1, l, st));
  DMD_TRY(dgemm(m, l, l, 1.0, Bs, m, false, b.T1, l, false, 0.0, b.WB, m, st));   // Bs R1^{-1}
  DMD_TRY(tall.nn(b.n, m, l, X, ldX, b.WB, b.Q1, b.ldY, b.gemm_ws, st));
  DMD_TRY(tall.tn(b.n, l, l, b.Q1, b.ldY, b.Q1, b.ldY, b.G, b.gemm_ws, st));
  DMD_TRY(cholesky_upper_f32(l, b.G, l, kTauTall, info, tag + 1, st));
  DMD_TRY(tri_inv_upper(l, b.G, l, b.T2, l, st));
  return orth_tall_shifted(tall, b, X, ldX, Bs, info, tag, st);
}

// One power iteration (Sec. 4.3) in the space of the snapshot Gram: with
// Q = X Bs R^{-1} the basis orth_tall would form from Bs (R = chol(Bs^T W_X
// Bs), the same first factor, with the same dropping rule and the same
// shifted fallback), X^T Q = W_X (Bs R^{-1}) exactly, so Z = X^T Q is formed
// from W_X = X^T X in FP64 and the tall basis is never built: the tall
// passes of an iteration (X Bs R^{-1} and X^T Q) become two m x m x l
// products.  The result is b.Z (m x l, not yet orthonormal); Bs may be b.Z.
dmd_status power_step_gram(FitBufs& b, const double* Bs, int32_t* info, int tag, cudaStream_t st) {
  const int l = b.l, m = b.m;
  const int32_t* skip = b.gate + 1;
  DMD_TRY(dgemm(m, l, m, 1.0, b.W, m + 1, false, Bs, m, false, 0.0, b.WB, m, st));
  DMD_TRY(dgemm(l, l, m, 1.0, Bs, m, true, b.WB, m, false, 0.0, b.G, l, st));
  DMD_TRY(fit_glue_copy((int64_t)l * l, b.G, b.G0, st));
  DMD_TRY(fit_glue_gate(info, b.gate, 0, 0, st));
  DMD_TRY(cholesky_upper(l, b.G, l, kTauTall, info, tag, st));
  DMD_TRY(fit_glue_gate(info, b.gate, 1, l - b.r, st));
  DMD_TRY(tri_inv_upper(l, b.G, l, b.T1, l, st));
  // more directions dropped than the sketch has spare: R = chol(G + s I)
  // instead (every direction kept), as the shifted fallback of orth_tall
  DMD_TRY(fit_glue_shift_diag(l, b.G0, l, 1e-6, skip, st));
  DMD_TRY(cholesky_upper_gated(l, b.G0, l, 0.0, info, tag + 2, skip, st));
  DMD_TRY(tri_inv_upper_gated(l, b.G0, l, b.T1, l, skip, st));
  DMD_TRY(dgemm(m, l, l, 1.0, Bs, m, false, b.T1, l, false, 0.0, b.WB, m, st));     // Bs R^{-1}
  DMD_TRY(dgemm(m, l, m, 1.0, b.W, m + 1, false, b.WB, m, false, 0.0, b.Z, m, st));  // X^T Q
  return DMD_OK;
}

// CholeskyQR2 of a small FP64 matrix Z (rows x l) in place (second factor in
// FP32, as for the tall sketch).
dmd_status orth_small(FitBufs& b, int rows, int32_t* info, int tag, cudaStream_t st) {
  const int l = b.l;
  for (int pass = 0; pass < 2; ++pass) {
    DMD_TRY(dgemm(l, l, rows, 1.0, b.Z, rows, true, b.Z, rows, false, 0.0, b.Gz, l, st));
    if (pass == 0) DMD_TRY(cholesky_upper(l, b.Gz, l, kTauSmall, info, tag + pass, st));
    else DMD_TRY(cholesky_upper_f32(l, b.Gz, l, kTauSmall, info, tag + pass, st));
    DMD_TRY(tri_inv_upper(l, b.Gz, l, b.Tz, l, st));
    DMD_TRY(dgemm(rows, l, l, 1.0, b.Z, rows, false, b.Tz, l, false, 0.0, b.Zp, rows, st));
    DMD_TRY(fit_glue_copy((int64_t)rows * l, b.Zp, b.Z, st));
  }
  return DMD_OK;
}

// Symmetric eigendecomposition H = Y diag(ev) Y^T (ev descending) of an n x n
// FP64 matrix: Householder tridiagonalisation, bisection, inverse iteration,
// back-transformation.  H is overwritten.
dmd_status sym_eig(int n, double* H, double* tau, double* ev, double* Y, double* scratch, cudaStream_t st) {
  DMD_TRY(sytrd(n, H, n, tau, st));
  DMD_TRY(tridiag_eig(n, H, n, ev, Y, scratch, st));
  DMD_TRY(apply_q(n, H, n, tau, Y, n, n, st));
  return DMD_OK;
}

// Eigendecomposition of the reduced operator A~ (r x r) into the modal layout:
// lam_re/lam_im (canonical order) and the real-form eigenvectors W_R.
dmd_status reduced_eig(FitBufs& b, double* modal, int32_t* info, cudaStream_t st) {
  const int r = b.r;
  DMD_TRY(fit_glue_copy((int64_t)r * r, b.At, b.Ah, st));
  DMD_TRY(fit_glue_maxabs((int64_t)r * r, b.At, b.hnorm, st));
  DMD_TRY(hessenberg(r, b.Ah, r, b.tauA, st));
  DMD_TRY(hqr(r, b.Ah, r, b.wr, b.wi, b.Hq, info, st));
  DMD_TRY(fit_glue_fill_int(r, b.heads, -1, st));
  DMD_TRY(collect_heads(r, b.wi, b.heads, b.nheads, info, st));
  DMD_CUDA_TRY(cudaMemsetAsync(b.Yre, 0, (size_t)r * r * sizeof(double), st));
  DMD_CUDA_TRY(cudaMemsetAsync(b.Yim, 0, (size_t)r * r * sizeof(double), st));
  DMD_TRY(hess_eigvecs(r, b.Ah, r, b.wr, b.wi, b.heads, r, b.Yre, b.Yim, b.invit, b.hnorm, st));
  DMD_TRY(apply_q(r, b.Ah, r, b.tauA, b.Yre, r, r, st));
  DMD_TRY(apply_q(r, b.Ah, r, b.tauA, b.Yim, r, r, st));
  DMD_TRY(normalize_complex(r, b.Yre, b.Yim, r, st));
  DMD_TRY(eig_layout(r, b.wr, b.wi, b.heads, b.nheads, b.Yre, b.Yim, b.WR, modal, modal + r, b.order, info, st));
  return DMD_OK;
}

// DMD with control (Eq. external_forces, with the unknown-B least-squares fit
// of [A B] from Omega = [X; Ups]) in the basis Q of the randomized range
// finder: B0 = Q^T X, B1 = Q^T X'.  Input space: SVD of [B0; Ups] truncated to
// p = r + q; output space U_hat: leading r left singular vectors of B1.
// A~ = U_hat^T B1 Vt St^-1 Ut1^T U_hat, modes Phi = X' Vt St^-1 Ut1^T U_hat W,
// amplitudes and real-form forcing by least squares:
// (B1 M) [beta | G_R] ~ [Q^T x_0 | B1 Vt St^-1 Ut2^T].
dmd_status fit_control(const dmd_fit_desc& d, const float* S, const float* Ups, float* PhiR, double* modal,
                       int32_t* info, const Tall& tall, FitBufs& b, cudaStream_t st) {
  const int m = b.m, l = b.l, r = b.r, q = b.q, L = b.L, pp = b.p;
  const double* B0 = b.P;
  const double* B1 = b.P + l;
  (void)B0;
  DMD_TRY(fit_glue_stack(l, q, m, b.P, Ups, b.Omc, st));
  DMD_TRY(dgemm(L, L, m, 1.0, b.Omc, L, false, b.Omc, L, true, 0.0, b.Hc, L, st));
  DMD_TRY(sym_eig(L, b.Hc, b.tauC, b.evC, b.YC, b.tridC, st));
  DMD_TRY(fit_glue_sigma_range(L, pp, b.evC, nullptr, b.invC, info, 7100, st));
  // Vt St^-1 = Omega_c^T Ut St^-2  (m x p)
  DMD_TRY(dgemm(m, pp, L, 1.0, b.Omc, L, true, b.YC, L, false, 0.0, b.VS, m, st));
  DMD_TRY(fit_glue_scale_cols(m, pp, b.VS, m, b.invC, st));
  // output space from B1 = Q^T X'
  DMD_TRY(dgemm(l, l, m, 1.0, B1, l, false, B1, l, true, 0.0, b.Hb, l, st));
  DMD_TRY(sym_eig(l, b.Hb, b.tauB, b.evB, b.YB, b.trid, st));
  DMD_TRY(fit_glue_sigma(l, r, b.evB, modal + 3 * r, b.invsq, info, st));
  // T1 = B1 Vt St^-1 (l x p); T2 = Ut1^T U_hat (p x r); Tmp = T1 T2; A~ = U_hat^T Tmp
  DMD_TRY(dgemm(l, pp, m, 1.0, B1, l, false, b.VS, m, false, 0.0, b.T1c, l, st));
  DMD_TRY(dgemm(pp, r, l, 1.0, b.YC, L, true, b.YB, l, false, 0.0, b.T2c, pp, st));
  DMD_TRY(dgemm(l, r, pp, 1.0, b.T1c, l, false, b.T2c, pp, false, 0.0, b.Tmp, l, st));
  DMD_TRY(dgemm(r, r, l, 1.0, b.YB, l, true, b.Tmp, l, false, 0.0, b.At, r, st));
  DMD_TRY(reduced_eig(b, modal, info, st));
  // modes: M_R = Vt St^-1 (T2 W_R)
  DMD_TRY(dgemm(pp, r, r, 1.0, b.T2c, pp, false, b.WR, r, false, 0.0, b.Tw, pp, st));
  DMD_TRY(dgemm(m, r, pp, 1.0, b.VS, m, false, b.Tw, pp, false, 0.0, b.MR, m, st));
  DMD_TRY(tall.nn(b.n, m, r, S + d.ldS, d.ldS, b.MR, PhiR, d.ldPhi, b.gemm_ws, st));
  // least squares for beta and G_R in the Q basis
  DMD_TRY(dgemm(l, r, r, 1.0, b.Tmp, l, false, b.WR, r, false, 0.0, b.LS, l, st));
  DMD_TRY(fit_glue_copy(l, b.P, b.rhsc, st));
  DMD_TRY(dgemm(l, q, pp, 1.0, b.T1c, l, false, b.YC + l, L, true, 0.0, b.rhsc + l, l, st));
  DMD_TRY(lstsq(l, r, b.LS, l, q + 1, b.rhsc, l, b.solc, r, info, st));
  DMD_TRY(fit_glue_copy(r, b.solc, modal + 2 * r, st));
  DMD_TRY(fit_glue_copy((int64_t)r * q, b.solc + r, modal + 4 * r, st));
  return DMD_OK;
}

// OptDMD request of fit_impl: options, stats output and its small-space buffers.
struct OptRequest {
  const dmd_optdmd_opts* opts;
  double* stats;
  OptBufs* bufs;
};

dmd_status fit_impl(const dmd_fit_desc& d, const float* S, const float* Ups, const double* Omega, float* PhiR,
                    double* modal, int32_t* info, FitBufs& b, cudaStream_t st, const OptRequest* opt = nullptr) {
  const StatusScope scope(info);   // bounded waits of this fit report to info
  const Tall tall{d.precision};
  const int64_t n = b.n;
  const int m = b.m, l = b.l, r = b.r, q = b.q;
  const float* X = S;
  const float* Xp = S + d.ldS;
  DMD_CUDA_TRY(cudaMemsetAsync(info, 0, DMD_INFO_WORDS * sizeof(int32_t), st));
  DMD_CUDA_TRY(cudaMemsetAsync(modal, 0, DMD_MODAL_DOUBLES(r, q) * sizeof(double), st));
  // 1. sketch test matrix (Sec. 4.3)
  if (Omega) {
    DMD_CUDA_TRY(cudaMemcpyAsync(b.Om, Omega, (size_t)m * l * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    DMD_TRY(launch_sketch(m, l, d.seed, b.Om, st));
  }
  // 2. snapshot Gram W = S^T S (one pass; also screens the input for NaN/Inf)
  DMD_TRY(tall.tn_accurate(n, m + 1, m + 1, S, d.ldS, S, d.ldS, b.W, b.gemm_ws, st));
  DMD_TRY(fit_glue_check_finite((int64_t)(m + 1) * (m + 1), b.W, info, 91, st));
  // 3-4. Y = X Omega, power iterations Z = orth(X^T Q), Y = X Z (in the
  // snapshot-Gram space), then Q = orth(Y) for the last Y
  const double* Bs = b.Om;
  for (int it = 0; it < d.power_iters; ++it) {
    DMD_TRY(power_step_gram(b, Bs, info, it == 0 ? 1 : 12 + 4 * (it - 1), st));
    DMD_TRY(orth_small(b, m, info, 10 + 4 * it, st));
    Bs = b.Z;
  }
  DMD_TRY(orth_tall(tall, b, X, d.ldS, Bs, info, d.power_iters == 0 ? 1 : 12 + 4 * (d.power_iters - 1), st));
  // 5. projection P = Q^T S = T2^T (Q1^T S): B = P[:, 0:m], Q^T X' = P[:, 1:m+1], Q^T x_0 = P[:, 0]
  DMD_TRY(tall.tn(n, l, m + 1, b.Q1, b.ldY, S, d.ldS, b.Pp, b.gemm_ws, st));
  DMD_TRY(dgemm(l, m + 1, l, 1.0, b.T2, l, true, b.Pp, l, false, 0.0, b.P, l, st));
  DMD_TRY(fit_glue_check_finite((int64_t)l * (m + 1), b.P, info, 90, st));
  if (q > 0) return fit_control(d, S, Ups, PhiR, modal, info, tall, b, st);
  const double* B = b.P;
  const double* Bp = b.P + l;
  // 5. SVD of B via B B^T = U_B Sigma^2 U_B^T (tridiagonalisation, bisection, inverse iteration)
  DMD_TRY(dgemm(l, l, m, 1.0, B, l, false, B, l, true, 0.0, b.Hb, l, st));
  DMD_TRY(sym_eig(l, b.Hb, b.tauB, b.evB, b.YB, b.trid, st));
  double* sigma = modal + 3 * r;
  DMD_TRY(fit_glue_sigma(l, r, b.evB, sigma, b.invsq, info, st));
  // 6. V Sigma^{-1} = B^T U_r Sigma^{-2}; reduced operator A~ = U_r^T (Q^T X') V Sigma^{-1} (Sec. 3.1)
  DMD_TRY(dgemm(m, r, l, 1.0, B, l, true, b.YB, l, false, 0.0, b.Vs, m, st));
  DMD_TRY(fit_glue_scale_cols(m, r, b.Vs, m, b.invsq, st));
  DMD_TRY(dgemm(l, r, m, 1.0, Bp, l, false, b.Vs, m, false, 0.0, b.Tmp, l, st));
  DMD_TRY(dgemm(r, r, l, 1.0, b.YB, l, true, b.Tmp, l, false, 0.0, b.At, r, st));
  // 7. eigendecomposition A~ W = W Lambda
  DMD_TRY(reduced_eig(b, modal, info, st));
  if (opt) {
    // OptDMD (Sec. 4.2) from these eigenvalues; modes Phi_R = Q1 (T2 U_B,r Wt)
    DMD_TRY(optdmd_small(m, r, l, B, b.YB, b.T2, modal, info, opt->stats, *opt->opts, *opt->bufs, st));
    return tall.nn(n, l, r, b.Q1, b.ldY, opt->bufs->Mlift, PhiR, d.ldPhi, b.gemm_ws, st);
  }
  // 8. modes Phi_R = X' M_R with M_R = V Sigma^{-1} W_R, and beside it (on a
  // side stream: one SM against a pass over X') 9. the amplitudes
  // min || (Q^T X') M_R beta - Q^T x_0 || (Eq. projection in the Q basis)
  DMD_TRY(dgemm(m, r, r, 1.0, b.Vs, m, false, b.WR, r, false, 0.0, b.MR, m, st));
  DMD_TRY(dgemm(l, r, r, 1.0, b.Tmp, l, false, b.WR, r, false, 0.0, b.LS, l, st));
  DMD_TRY(fit_glue_copy(l, b.P, b.rhs, st));
  const Side* sd = side_of(st);
  cudaStream_t ss = st;
  if (sd) {
    DMD_CUDA_TRY(cudaEventRecord(sd->fork, st));
    DMD_CUDA_TRY(cudaStreamWaitEvent(sd->side, sd->fork, 0));
    ss = sd->side;
  }
  const dmd_status ls = lstsq(l, r, b.LS, l, 1, b.rhs, l, modal + 2 * r, r, info, ss);
  const dmd_status md = ls == DMD_OK ? tall.nn(n, m, r, Xp, d.ldS, b.MR, PhiR, d.ldPhi, b.gemm_ws, st, sd ? 1 : 0) : ls;
  if (sd) {   // join even after a failure, so the caller's stream covers all queued work
    DMD_CUDA_TRY(cudaEventRecord(sd->join, sd->side));
    DMD_CUDA_TRY(cudaStreamWaitEvent(st, sd->join, 0));
  }
  return md;
}

// ------------------------------------------------------------ predict layout

struct PredBufs {
  double *C, *Xi, *dC, *dXi, *Mu, *partial;
  float* F;
  void* gemm_ws;
};

int chunk_of(const dmd_predict_desc& d) { return d.chunk > 0 ? d.chunk : 50; }

// The streamed loss runs on the tensor cores with the frames kept on chip
// (mixed form, r <= 160); otherwise frames are recomputed in stored chunks.
bool fused_loss(const dmd_predict_desc& d) {
  return d.precision == DMD_MIXED_BF16X3 && umma_loss_grad_supported(d.r);
}

void carve_predict(Arena& a, const dmd_predict_desc& d, int mode, PredBufs& b) {
  // mode 0: forward, 1: backward from dOut, 2: streamed loss, 3: streamed
  // loss and its gradient
  const Tall tall{d.precision};
  const int r = d.r, K = d.K;
  const int steps = d.q > 0 ? d.steps : 0;
  const bool grad = mode == 1 || mode == 3, loss = mode >= 2;
  b.C = a.take<double>((size_t)r * K);
  b.Xi = a.take<double>((size_t)r * (steps + 1));
  b.dC = grad ? a.take<double>((size_t)r * K) : nullptr;
  b.dXi = grad ? a.take<double>((size_t)r * (steps + 1)) : nullptr;
  b.Mu = grad ? a.take<double>((size_t)r * (steps + 1)) : nullptr;
  b.partial = loss ? a.take<double>((size_t)std::max(loss_blocks(), umma_loss_parts(d.n))) : nullptr;
  const bool fused = loss && fused_loss(d);
  const int ch = std::min(chunk_of(d), K);
  b.F = (loss && !fused) ? a.take<float>((size_t)round_up(d.n, 32) * ch) : nullptr;
  size_t g = 0;
  if (mode == 0) g = tall.nn_bytes(d.n, r, K);
  if (mode == 1) g = tall.tn_bytes(d.n, r, K);
  if (mode == 2 && fused) g = umma_nn_workspace_bytes(d.n, r, std::min(K, 4096));
  if (mode == 3 && fused) g = umma_loss_grad_workspace_bytes(d.n, r, K);
  if (mode == 2 && !fused) g = tall.nn_bytes(d.n, r, ch);
  if (mode == 3 && !fused) g = std::max(tall.nn_bytes(d.n, r, ch), tall.tn_bytes(d.n, r, ch));
  b.gemm_ws = a.take<char>(g, 1024);
}

dmd_status validate_predict(const dmd_predict_desc* d, bool need_out_ld) {
  DMD_REQUIRE(d != nullptr, "predict: desc is NULL");
  DMD_REQUIRE(d->n >= 1 && d->r >= 1 && d->r <= 512 && d->K >= 1, "predict: need n >= 1, 1 <= r <= 512, K >= 1");
  DMD_REQUIRE(d->ldPhi >= d->n && d->ldPhi % 4 == 0, "predict: ldPhi must be >= n and a multiple of 4");
  if (need_out_ld) DMD_REQUIRE(d->ldOut >= d->n && d->ldOut % 4 == 0, "predict: ldOut must be >= n and a multiple of 4");
  DMD_REQUIRE(d->q >= 0 && d->q <= 64, "predict: q must be in [0, 64]");
  DMD_REQUIRE(d->q == 0 || d->steps >= 0, "predict: steps must be >= 0 with control");
  DMD_REQUIRE(valid_precision(d->precision), "predict: unknown precision %d", d->precision);
  return DMD_OK;
}

dmd_status form_coefficients(const dmd_predict_desc& d, const double* modal, const int32_t* k, const float* u,
                             PredBufs& b, cudaStream_t st) {
  if (d.q > 0) {
    DMD_TRY(launch_rollout(d.r, d.q, d.steps, modal, u, b.Xi, st));
    DMD_TRY(launch_gather_cols(d.r, d.K, b.Xi, k, d.steps, b.C, nullptr, st));
  } else {
    DMD_TRY(launch_coefficients(d.r, d.K, modal, k, b.C, st));
  }
  return DMD_OK;
}

dmd_status chain_rule(const dmd_predict_desc& d, const double* modal, const int32_t* k, const float* u,
                      double* d_modal, float* d_u, PredBufs& b, cudaStream_t st) {
  DMD_CUDA_TRY(cudaMemsetAsync(d_modal, 0, DMD_MODAL_DOUBLES(d.r, d.q) * sizeof(double), st));
  if (d.q > 0) {
    DMD_TRY(launch_rollout(d.r, d.q, d.steps, modal, u, b.Xi, st));
    DMD_TRY(launch_rollout_adjoint(d.r, d.q, d.steps, d.K, k, modal, u, b.Xi, b.dC, b.dXi, b.Mu, d_modal, d_u,
                                   st));
  } else {
    DMD_TRY(launch_chain_closed(d.r, d.K, modal, k, b.dC, d_modal, st));
  }
  return DMD_OK;
}

template <class F>
dmd_status with_arena(void* ws, size_t ws_bytes, F&& carve_and_run, size_t need) {
  if (ws_bytes < need) {
    set_error("workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
    return DMD_ENOMEM;
  }
  DMD_REQUIRE(ws != nullptr, "workspace is NULL");
  DMD_REQUIRE(((uintptr_t)ws & 255) == 0, "workspace must be 256-byte aligned");
  Arena a{reinterpret_cast<char*>(ws), ws_bytes, 0};
  return carve_and_run(a);
}

// ------------------------------------------------------------ upsampling

struct UpBufs {
  double *G, *Pin, *P, *C;
  void* gemm_ws;
};

void carve_upsample(Arena& a, const dmd_upsample_desc& d, UpBufs& b) {
  const Tall tall{d.precision};
  const int r = d.r, T = d.T;
  b.G = a.take<double>((size_t)r * r);
  b.Pin = a.take<double>((size_t)r * (T + 1));
  b.P = a.take<double>((size_t)r * (T + 1));
  b.C = a.take<double>((size_t)r * T);
  size_t g = tall.tn_accurate_bytes(d.n, r, r);
  g = std::max(g, tall.tn_bytes(d.n, r, T + 1));
  g = std::max(g, tall.nn_bytes(d.n, r, T));
  b.gemm_ws = a.take<char>(g, 1024);
}

dmd_status validate_upsample(const dmd_upsample_desc* d) {
  DMD_REQUIRE(d != nullptr, "dmd_upsample: desc is NULL");
  DMD_REQUIRE(d->n >= 1 && d->r >= 1 && d->r <= 200 && d->T >= 1 && d->r <= d->n,
              "dmd_upsample: need n >= 1, 1 <= r <= min(200, n), T >= 1 (got n=%lld r=%d T=%d)", (long long)d->n,
              d->r, d->T);
  DMD_REQUIRE(d->ldPhi >= d->n && d->ldIn >= d->n && d->ldOut >= d->n && d->ldPhi % 4 == 0 && d->ldIn % 4 == 0 &&
                  d->ldOut % 4 == 0,
              "dmd_upsample: leading dimensions must be >= n and multiples of 4");
  DMD_REQUIRE(valid_precision(d->precision), "dmd_upsample: bad precision %d", d->precision);
  DMD_REQUIRE(d->dt > 0.0 && d->threshold >= 0.0, "dmd_upsample: need dt > 0 and threshold >= 0");
  DMD_REQUIRE(d->gram_given == 0 || d->gram_given == 1, "dmd_upsample: gram_given must be 0 or 1");
  return DMD_OK;
}

// ------------------------------------------------------ density advection

struct AdvBufs {
  int32_t* ks;
  double* C;
  float* U;
  int64_t ldU;
  int ch;
  void* gemm_ws;
};

int64_t cells_of(const dmd_advect_desc& d) {
  int64_t c = 1;
  for (int i = 0; i < d.dim; ++i) c *= d.N;
  return c;
}

void carve_advect(Arena& a, const dmd_advect_desc& d, AdvBufs& b) {
  const Tall tall{d.precision};
  const int64_t n = d.dim * cells_of(d);
  b.ch = std::min(d.chunk > 0 ? d.chunk : 256, d.K);
  b.ldU = round_up(n, 32);
  b.ks = a.take<int32_t>(b.ch);
  b.C = a.take<double>((size_t)d.r * b.ch);
  b.U = a.take<float>((size_t)b.ldU * b.ch, 1024);
  b.gemm_ws = a.take<char>(tall.nn_bytes(n, d.r, b.ch), 1024);
}

dmd_status validate_advect(const dmd_advect_desc* d) {
  DMD_REQUIRE(d != nullptr, "dmd_advect_density: desc is NULL");
  DMD_REQUIRE((d->dim == 2 || d->dim == 3) && d->N >= 2 && d->N <= (d->dim == 2 ? 32768 : 1024) && d->r >= 1 &&
                  d->K >= 1,
              "dmd_advect_density: need dim 2 or 3, 2 <= N <= 32768 (2D) or 1024 (3D), r >= 1, K >= 1 "
              "(got dim=%d N=%d r=%d K=%d)", d->dim, d->N, d->r, d->K);
  const int64_t cells = cells_of(*d);
  DMD_REQUIRE(d->ldPhi >= d->dim * cells && d->ldRho >= cells && d->ldPhi % 4 == 0 && d->ldRho % 4 == 0,
              "dmd_advect_density: leading dimensions must cover the grid and be multiples of 4");
  DMD_REQUIRE(valid_precision(d->precision) && d->chunk >= 0, "dmd_advect_density: bad precision or chunk");
  DMD_REQUIRE(std::isfinite(d->dt), "dmd_advect_density: dt must be finite");
  return DMD_OK;
}

}  // namespace
}  // namespace dmd

using namespace dmd;

extern "C" dmd_status dmd_advect_workspace_bytes(const dmd_advect_desc* desc, size_t* bytes) {
  DMD_TRY(validate_advect(desc));
  DMD_REQUIRE(bytes != nullptr, "bytes is NULL");
  Arena a;
  AdvBufs b;
  carve_advect(a, *desc, b);
  *bytes = a.used + 256;
  return DMD_OK;
}

extern "C" dmd_status dmd_advect_density(const dmd_advect_desc* desc, const float* Phi_R, const double* modal,
                                         const float* rho0, float* rho, void* workspace, size_t ws_bytes,
                                         void* stream) {
  size_t need = 0;
  DMD_TRY(dmd_advect_workspace_bytes(desc, &need));
  DMD_REQUIRE(Phi_R && modal && rho0 && rho, "dmd_advect_density: NULL pointer argument");
  const dmd_advect_desc& d = *desc;
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    AdvBufs b;
    carve_advect(a, d, b);
    const Tall tall{d.precision};
    const int64_t cells = cells_of(d), n = d.dim * cells;
    DMD_CUDA_TRY(cudaMemcpyAsync(rho, rho0, (size_t)cells * sizeof(float), cudaMemcpyDeviceToDevice, st));
    for (int k0 = 0; k0 < d.K; k0 += b.ch) {
      const int c = std::min(b.ch, d.K - k0);
      DMD_TRY(launch_iota(b.ks, c, k0, st));
      DMD_TRY(launch_coefficients(d.r, c, modal, b.ks, b.C, st));
      DMD_TRY(tall.nn(n, d.r, c, Phi_R, d.ldPhi, b.C, b.U, b.ldU, b.gemm_ws, st));
      for (int j = 0; j < c; ++j) {
        const int k = k0 + j;
        DMD_TRY(launch_advect(d.dim, d.N, rho + (int64_t)k * d.ldRho, rho + (int64_t)(k + 1) * d.ldRho,
                              b.U + (int64_t)j * b.ldU, (float)d.dt, st));
      }
    }
    return DMD_OK;
  }, need);
}

extern "C" dmd_status dmd_upsample_workspace_bytes(const dmd_upsample_desc* desc, size_t* bytes) {
  DMD_TRY(validate_upsample(desc));
  DMD_REQUIRE(bytes != nullptr, "bytes is NULL");
  Arena a;
  UpBufs b;
  carve_upsample(a, *desc, b);
  *bytes = a.used + 256;
  return DMD_OK;
}

// Sec. 6.3.1: G = Phi_R^T Phi_R (FP32 products, FP64 sums, both forms: its
// Cholesky factor turns Phi_R^T [H_0 | L] into the least-squares coordinates),
// P = G^{-1} Phi_R^T [H_0 | L], C from P (closed-form evolution of the
// high-order modes), out = Phi_R C.
extern "C" dmd_status dmd_upsample(const dmd_upsample_desc* desc, const float* Phi_R, const double* modal,
                                   const float* in, float* out, double* gram, int32_t* info, void* workspace,
                                   size_t ws_bytes, void* stream) {
  size_t need = 0;
  DMD_TRY(dmd_upsample_workspace_bytes(desc, &need));
  DMD_REQUIRE(Phi_R && modal && in && out && info, "dmd_upsample: NULL pointer argument");
  DMD_REQUIRE(desc->gram_given == 0 || gram != nullptr, "dmd_upsample: gram_given needs gram");
  const dmd_upsample_desc& d = *desc;
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    UpBufs b;
    carve_upsample(a, d, b);
    const Tall tall{d.precision};
    const int r = d.r, T = d.T;
    const StatusScope scope(info);
    DMD_CUDA_TRY(cudaMemsetAsync(info, 0, DMD_INFO_WORDS * sizeof(int32_t), st));
    if (d.gram_given) {
      DMD_CUDA_TRY(cudaMemcpyAsync(b.G, gram, (size_t)r * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      DMD_TRY(tall.tn_accurate(d.n, r, r, Phi_R, d.ldPhi, Phi_R, d.ldPhi, b.G, b.gemm_ws, st));
      if (gram) {
        DMD_CUDA_TRY(cudaMemcpyAsync(gram, b.G, (size_t)r * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
    }
    DMD_TRY(tall.tn(d.n, r, T + 1, Phi_R, d.ldPhi, in, d.ldIn, b.Pin, b.gemm_ws, st));
    DMD_TRY(cholesky_upper(r, b.G, r, 1e-13, info, 95, st));
    DMD_TRY(chol_solve_gated(r, b.G, r, b.Pin, r, T + 1, 1.0, 0.0, b.P, r, nullptr, st));
    DMD_TRY(launch_upsample_coeffs(r, T, modal, d.threshold, d.dt, b.P, b.C, st));
    return tall.nn(d.n, r, T, Phi_R, d.ldPhi, b.C, out, d.ldOut, b.gemm_ws, st);
  }, need);
}

extern "C" {

const char* dmd_last_error(void) { return g_err; }
const char* dmd_version(void) { return "libdmd 0.1 (sm_103a)"; }
uint64_t dmd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

dmd_status dmd_async_status(int32_t* words, int32_t clear, void* stream) {
  DMD_REQUIRE(words != nullptr, "dmd_async_status: words is NULL");
  int32_t* w = async_status_word();
  DMD_REQUIRE(w != nullptr, "dmd_async_status: no status word on the current device");
  cudaStream_t st = (cudaStream_t)stream;
  DMD_CUDA_TRY(cudaMemcpyAsync(words, w, DMD_INFO_WORDS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (clear) DMD_CUDA_TRY(cudaMemsetAsync(w, 0, DMD_INFO_WORDS * sizeof(int32_t), st));
  DMD_CUDA_TRY(cudaStreamSynchronize(st));
  return DMD_OK;
}

dmd_status dmd_fit_workspace_bytes(const dmd_fit_desc* desc, size_t* bytes) {
  DMD_TRY(validate_fit(desc));
  DMD_REQUIRE(bytes != nullptr, "bytes is NULL");
  Arena a;
  FitBufs b;
  carve_fit(a, *desc, Tall{desc->precision}, b);
  *bytes = a.used + 256;
  return DMD_OK;
}

dmd_status dmd_fit(const dmd_fit_desc* desc, const float* S, const float* Ups, const double* Omega, float* Phi_R,
                   double* modal, int32_t* info, void* workspace, size_t ws_bytes, void* stream) {
  DMD_TRY(validate_fit(desc));
  DMD_REQUIRE(S && Phi_R && modal && info, "dmd_fit: NULL pointer argument");
  DMD_REQUIRE(desc->q == 0 || Ups != nullptr, "dmd_fit: q > 0 needs Ups");
  size_t need = 0;
  DMD_TRY(dmd_fit_workspace_bytes(desc, &need));
  return with_arena(workspace, ws_bytes, [&](Arena& a) {
    FitBufs b;
    carve_fit(a, *desc, Tall{desc->precision}, b);
    return fit_impl(*desc, S, Ups, Omega, Phi_R, modal, info, b, (cudaStream_t)stream);
  }, need);
}

dmd_status dmd_fit_optdmd_workspace_bytes(const dmd_fit_desc* desc, size_t* bytes) {
  DMD_TRY(validate_fit(desc));
  DMD_REQUIRE(bytes != nullptr, "bytes is NULL");
  DMD_REQUIRE(desc->q == 0, "dmd_fit_optdmd: control inputs (q > 0) are not supported");
  DMD_REQUIRE(desc->r <= 200, "dmd_fit_optdmd: r = %d above 200 (the small solver's factor lives in shared memory)",
              desc->r);
  Arena a;
  FitBufs b;
  carve_fit(a, *desc, Tall{desc->precision}, b);
  OptBufs o;
  carve_optdmd(a, desc->m, desc->r, b.l, o);
  *bytes = a.used + 256;
  return DMD_OK;
}

dmd_status dmd_fit_optdmd(const dmd_fit_desc* desc, const dmd_optdmd_opts* opts, const float* S,
                          const double* Omega, float* Phi_R, double* modal, int32_t* info, double* stats,
                          void* workspace, size_t ws_bytes, void* stream) {
  size_t need = 0;
  DMD_TRY(dmd_fit_optdmd_workspace_bytes(desc, &need));
  DMD_REQUIRE(S && Phi_R && modal && info, "dmd_fit_optdmd: NULL pointer argument");
  dmd_optdmd_opts o{};
  if (opts) o = *opts;
  DMD_REQUIRE(o.max_evals >= 0 && o.tol >= 0.0 && o.mu0 >= 0.0 && o.max_evals <= 10000,
              "dmd_fit_optdmd: bad options (max_evals %d, tol %g, mu0 %g)", o.max_evals, o.tol, o.mu0);
  return with_arena(workspace, ws_bytes, [&](Arena& a) {
    FitBufs b;
    carve_fit(a, *desc, Tall{desc->precision}, b);
    OptBufs ob;
    carve_optdmd(a, desc->m, desc->r, b.l, ob);
    OptRequest req{&o, stats, &ob};
    return fit_impl(*desc, S, nullptr, Omega, Phi_R, modal, info, b, (cudaStream_t)stream, &req);
  }, need);
}

dmd_status dmd_predict_workspace_bytes(const dmd_predict_desc* desc, size_t* bytes) {
  DMD_TRY(validate_predict(desc, false));
  DMD_REQUIRE(bytes != nullptr, "bytes is NULL");
  size_t best = 0;
  for (int mode = 0; mode < 2; ++mode) {
    Arena a;
    PredBufs b;
    carve_predict(a, *desc, mode, b);
    best = std::max(best, a.used + 256);
  }
  *bytes = best;
  return DMD_OK;
}

dmd_status dmd_predict_loss_workspace_bytes(const dmd_predict_desc* desc, int32_t want_grad, size_t* bytes) {
  DMD_TRY(validate_predict(desc, false));
  DMD_REQUIRE(bytes != nullptr, "bytes is NULL");
  Arena a;
  PredBufs b;
  carve_predict(a, *desc, want_grad ? 3 : 2, b);
  *bytes = a.used + 256;
  return DMD_OK;
}

dmd_status dmd_predict(const dmd_predict_desc* desc, const float* Phi_R, const double* modal, const int32_t* k,
                       const float* u, float* out, void* workspace, size_t ws_bytes, void* stream) {
  DMD_TRY(validate_predict(desc, true));
  DMD_REQUIRE(Phi_R && modal && k && out, "dmd_predict: NULL pointer argument");
  DMD_REQUIRE(desc->q == 0 || u != nullptr || desc->steps == 0, "dmd_predict: q > 0 needs u");
  size_t need = 0;
  DMD_TRY(dmd_predict_workspace_bytes(desc, &need));
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    PredBufs b;
    carve_predict(a, *desc, 0, b);
    DMD_TRY(form_coefficients(*desc, modal, k, u, b, st));
    const Tall tall{desc->precision};
    return tall.nn(desc->n, desc->r, desc->K, Phi_R, desc->ldPhi, b.C, out, desc->ldOut, b.gemm_ws, st);
  }, need);
}

dmd_status dmd_predict_backward(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                                const int32_t* k, const float* u, const float* dOut, double* d_modal, float* d_u,
                                void* workspace, size_t ws_bytes, void* stream) {
  DMD_TRY(validate_predict(desc, true));
  DMD_REQUIRE(Phi_R && modal && k && dOut && d_modal, "dmd_predict_backward: NULL pointer argument");
  size_t need = 0;
  DMD_TRY(dmd_predict_workspace_bytes(desc, &need));
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    PredBufs b;
    carve_predict(a, *desc, 1, b);
    const Tall tall{desc->precision};
    DMD_TRY(tall.tn(desc->n, desc->r, desc->K, Phi_R, desc->ldPhi, dOut, desc->ldOut, b.dC, b.gemm_ws, st));
    return chain_rule(*desc, modal, k, u, d_modal, d_u, b, st);
  }, need);
}

dmd_status dmd_predict_loss(const dmd_predict_desc* desc, const float* Phi_R, const double* modal, const int32_t* k,
                            const float* u, const float* target, const double* w, const dmd_loss_opts* opts,
                            int32_t want_grad, double* loss, double* d_modal, float* d_u, void* workspace,
                            size_t ws_bytes, void* stream) {
  DMD_TRY(validate_predict(desc, false));
  DMD_REQUIRE(Phi_R && modal && k && target && w && loss, "dmd_predict_loss: NULL pointer argument");
  DMD_REQUIRE(!want_grad || d_modal, "dmd_predict_loss: want_grad needs d_modal");
  DMD_REQUIRE(opts == nullptr || opts->kind == DMD_LOSS_QUADRATIC ||
                  (opts->kind == DMD_LOSS_HUBER && std::isfinite(opts->delta) && opts->delta > 0.0),
              "dmd_predict_loss: loss kind must be quadratic or Huber with a finite delta > 0");
  const float delta = (opts && opts->kind == DMD_LOSS_HUBER) ? (float)opts->delta : 0.f;
  size_t need = 0;
  DMD_TRY(dmd_predict_loss_workspace_bytes(desc, want_grad, &need));
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    PredBufs b;
    carve_predict(a, *desc, want_grad ? 3 : 2, b);
    const Tall tall{desc->precision};
    DMD_TRY(form_coefficients(*desc, modal, k, u, b, st));
    if (fused_loss(*desc)) {
      int parts = 0;
      if (want_grad)
        DMD_TRY(umma_loss_grad(desc->n, desc->r, desc->K, Phi_R, desc->ldPhi, b.C, target, w, delta, b.dC, b.partial,
                               &parts, b.gemm_ws, st));
      if (want_grad) {
        DMD_TRY(launch_sum_partials(parts, b.partial, loss, false, st));
      } else {
        // the loss kernel stages the frames' weights in shared memory: at
        // most 4096 frames per launch
        for (int j0 = 0; j0 < desc->K; j0 += 4096) {
          const int nf = std::min(4096, desc->K - j0);
          DMD_TRY(umma_loss_nn(desc->n, desc->r, nf, Phi_R, desc->ldPhi, b.C + (size_t)j0 * desc->r, target, w + j0,
                               delta, b.partial, &parts, b.gemm_ws, st));
          DMD_TRY(launch_sum_partials(parts, b.partial, loss, j0 > 0, st));
        }
      }
    } else {
      const int ch = std::min(chunk_of(*desc), desc->K);
      const int64_t ldF = round_up(desc->n, 32);
      for (int j0 = 0; j0 < desc->K; j0 += ch) {
        const int nf = std::min(ch, desc->K - j0);
        DMD_TRY(tall.nn(desc->n, desc->r, nf, Phi_R, desc->ldPhi, b.C + (size_t)j0 * desc->r, b.F, ldF, b.gemm_ws,
                        st));
        DMD_TRY(launch_loss_chunk(desc->n, nf, b.F, ldF, target, w + j0, want_grad != 0, delta, b.partial, loss,
                                  j0 > 0, st));
        if (want_grad)
          DMD_TRY(tall.tn(desc->n, desc->r, nf, Phi_R, desc->ldPhi, b.F, ldF, b.dC + (size_t)j0 * desc->r,
                          b.gemm_ws, st));
      }
    }
    if (want_grad) return chain_rule(*desc, modal, k, u, d_modal, d_u, b, st);
    return DMD_OK;
  }, need);
}

dmd_status dmd_sketch_matrix(int32_t m, int32_t l, uint64_t seed, double* Omega, void* stream) {
  DMD_REQUIRE(m >= 1 && l >= 1 && Omega, "dmd_sketch_matrix: bad arguments");
  return launch_sketch(m, l, seed, Omega, (cudaStream_t)stream);
}

dmd_status dmd_philox_blocks(int64_t count, uint32_t stream_id, uint64_t key, uint32_t* out, void* stream) {
  DMD_REQUIRE(count >= 0 && (count == 0 || out), "dmd_philox_blocks: bad arguments");
  DMD_REQUIRE(((uintptr_t)out & 15) == 0, "dmd_philox_blocks: out must be 16-byte aligned");
  return launch_philox_blocks(count, stream_id, key, out, (cudaStream_t)stream);
}

dmd_status dmd_gemm_tall_workspace_bytes(int32_t precision, int64_t n, int32_t Kd, int32_t N, size_t* bytes) {
  DMD_REQUIRE(valid_precision(precision) && n >= 1 && Kd >= 1 && N >= 1 && bytes, "gemm_tall: bad arguments");
  *bytes = Tall{precision}.nn_bytes(n, Kd, N) + 1024;
  return DMD_OK;
}

dmd_status dmd_gemm_tall(int32_t precision, int64_t n, int32_t Kd, int32_t N, const float* A, int64_t lda,
                         const double* B, float* C, int64_t ldc, double* gram, void* workspace, size_t ws_bytes,
                         void* stream) {
  DMD_REQUIRE(valid_precision(precision) && n >= 1 && Kd >= 1 && N >= 1, "gemm_tall: bad sizes");
  DMD_REQUIRE(Kd <= 1024 && N <= 65536, "gemm_tall: Kd <= 1024 and N <= 65536");
  DMD_REQUIRE(A && B && C, "gemm_tall: NULL pointer");
  DMD_REQUIRE(lda >= n && lda % 4 == 0 && ldc >= n && ldc % 4 == 0, "gemm_tall: lda/ldc must be >= n, multiple of 4");
  const Tall tall{precision};
  size_t need = tall.nn_bytes(n, Kd, N) + 1024;
  if (gram) need = std::max(need, tall.tn_bytes(n, N, N) + 1024);
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    void* ws = a.take<char>(ws_bytes - 1024, 1024);
    DMD_TRY(tall.nn(n, Kd, N, A, lda, B, C, ldc, ws, st));
    if (gram) DMD_TRY(tall.tn(n, N, N, C, ldc, C, ldc, gram, ws, st));
    return DMD_OK;
  }, need);
}

dmd_status dmd_gemm_tn_workspace_bytes(int32_t precision, int64_t n, int32_t Ka, int32_t N, size_t* bytes) {
  DMD_REQUIRE(valid_precision(precision) && n >= 1 && Ka >= 1 && N >= 1 && bytes, "gemm_tn: bad arguments");
  *bytes = Tall{precision}.tn_bytes(n, Ka, N) + 1024;
  return DMD_OK;
}

dmd_status dmd_gemm_tn(int32_t precision, int64_t n, int32_t Ka, int32_t N, const float* A, int64_t lda,
                       const float* B, int64_t ldb, double* C, void* workspace, size_t ws_bytes, void* stream) {
  DMD_REQUIRE(valid_precision(precision) && n >= 1 && Ka >= 1 && N >= 1, "gemm_tn: bad sizes");
  DMD_REQUIRE(Ka <= 1024 && N <= 65536, "gemm_tn: Ka <= 1024 and N <= 65536");
  DMD_REQUIRE(A && B && C, "gemm_tn: NULL pointer");
  DMD_REQUIRE(lda >= n && lda % 4 == 0 && ldb >= n && ldb % 4 == 0, "gemm_tn: lda/ldb must be >= n, multiple of 4");
  const Tall tall{precision};
  const size_t need = tall.tn_bytes(n, Ka, N) + 1024;
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    void* ws = a.take<char>(ws_bytes - 1024, 1024);
    return tall.tn(n, Ka, N, A, lda, B, ldb, C, ws, st);
  }, need);
}

}  // extern "C"

extern "C" dmd_status dmd_edit_modes(int32_t r, int32_t q, const double* modal_in, double* modal_out,
                                     double threshold, const double* low, const double* high, double dt,
                                     void* stream) {
  DMD_REQUIRE(r >= 1 && q >= 0 && modal_in && modal_out && low && high, "dmd_edit_modes: bad arguments");
  DMD_REQUIRE(dt > 0.0 && threshold >= 0.0, "dmd_edit_modes: need dt > 0 and threshold >= 0");
  DMD_REQUIRE(modal_in != modal_out, "dmd_edit_modes: modal_out must not alias modal_in");
  return launch_edit_modes(r, q, modal_in, modal_out, threshold, low, high, dt, (cudaStream_t)stream);
}

extern "C" dmd_status dmd_autotune_predict(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                                           const int32_t* k, float* out, void* workspace, size_t ws_bytes,
                                           void* stream, int32_t* chosen) {
  DMD_TRY(validate_predict(desc, true));
  DMD_REQUIRE(Phi_R && modal && k && out, "dmd_autotune_predict: NULL pointer argument");
  DMD_REQUIRE(desc->q == 0, "dmd_autotune_predict: tune without control inputs");
  size_t need = 0;
  DMD_TRY(dmd_predict_workspace_bytes(desc, &need));
  cudaStream_t st = (cudaStream_t)stream;
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    PredBufs b;
    carve_predict(a, *desc, 0, b);
    DMD_TRY(form_coefficients(*desc, modal, k, nullptr, b, st));
    if (desc->precision != DMD_MIXED_BF16X3) {
      if (chosen) chosen[0] = chosen[1] = chosen[2] = 0;
      return DMD_OK;
    }
    return umma_tune_nn(desc->n, desc->r, desc->K, Phi_R, desc->ldPhi, b.C, out, desc->ldOut, b.gemm_ws, st, chosen);
  }, need);
}

namespace dmd {

// Forward prediction with a workspace sized for the forward pass alone (the
// coefficient matrix, the control rollout and the tall product's scratch);
// dmd_predict_workspace_bytes covers the backward and loss passes as well.
// Used by dmd_predict_noalloc, whose workspace is a fixed device array, and
// by the batch driver; `who` names the caller's entry point in error messages.
dmd_status predict_forward_workspace_bytes(const dmd_predict_desc* desc, size_t* bytes) {
  DMD_TRY(validate_predict(desc, true));
  Arena a;
  PredBufs b;
  carve_predict(a, *desc, 0, b);
  *bytes = a.used + 256;
  return DMD_OK;
}

dmd_status predict_forward(const dmd_predict_desc* desc, const float* Phi_R, const double* modal, const int32_t* k,
                           const float* u, float* out, void* workspace, size_t ws_bytes, cudaStream_t st,
                           const char* who) {
  DMD_TRY(validate_predict(desc, true));
  DMD_REQUIRE(Phi_R && modal && k && out, "%s: NULL pointer argument", who);
  DMD_REQUIRE(desc->q == 0 || u != nullptr || desc->steps == 0, "%s: q > 0 needs u", who);
  size_t need = 0;
  DMD_TRY(predict_forward_workspace_bytes(desc, &need));
  return with_arena(workspace, ws_bytes, [&](Arena& a) -> dmd_status {
    PredBufs b;
    carve_predict(a, *desc, 0, b);
    DMD_TRY(form_coefficients(*desc, modal, k, u, b, st));
    const Tall tall{desc->precision};
    return tall.nn(desc->n, desc->r, desc->K, Phi_R, desc->ldPhi, b.C, out, desc->ldOut, b.gemm_ws, st);
  }, need);
}

}  // namespace dmd
