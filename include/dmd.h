/*
 * libdmd -- C ABI of the GB300 (sm_103a) DMD / DMDc hot path.
 *
 * Method: "Fast Subspace Fluid Simulation with a Temporally-Aware Basis"
 * (arXiv 2502.05339).  The library fits an exact DMD operator from a tall
 * snapshot matrix through a randomized SVD (Sec. 3.1, Sec. 4.3, Sec. 4.6) and
 * predicts many time points at once by exponential integration
 * u(t + k dt) = Phi Lambda^k z(t) (Eq. large_time_step), with a hand-written
 * adjoint of the prediction.  On top of the fit and the prediction: the
 * OptDMD fit (Sec. 4.2), temporal editing (Eq. edit_temporal), upsampling
 * evolution (Sec. 6.3.1), density advection in the model's velocity
 * (Sec. 7.2) and a batched many-scene driver.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major.  A tall matrix with n rows uses a leading
 *   dimension ld >= n with ld % 4 == 0 (16-byte column starts, as TMA needs).
 * - Every pointer argument is a DEVICE pointer unless stated otherwise.  The
 *   caller owns all memory (inputs, outputs, workspace); the library never
 *   allocates or frees device memory and keeps no pointer after the stream
 *   work it enqueued has finished.
 * - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL
 *   for the legacy default stream).  The return value reports argument errors
 *   (DMD_EINVAL), a workspace that is too small (DMD_ENOMEM) and launch
 *   failures (DMD_ECUDA).  Failures found on the device (numerical breakdown,
 *   rank deficiency, non-finite input, a bounded wait that ran out) are
 *   written to the device status word info[0]; read it after synchronising.
 * - No C++ exception crosses this boundary.  dmd_last_error() returns a
 *   thread-local description of the last host-side failure.
 * - Precision: DMD_FP32 runs the passes over the snapshots in plain FP32 on
 *   the CUDA cores; DMD_MIXED_BF16X3 runs them on the tcgen05 tensor cores
 *   with every FP32 operand split into bf16 hi + lo and the products
 *   hi*hi + hi*lo + lo*hi accumulated in FP32.  The small dense solvers
 *   (Cholesky, SVD of B, the reduced operator, its eigendecomposition, the
 *   least-squares amplitudes) run in FP64 in both forms.
 *
 * Real 2x2-block model layout ("modal" buffer, FP64, device)
 * -----------------------------------------------------------
 * For rank r and q control channels the model occupies DMD_MODAL_DOUBLES(r, q)
 * doubles:
 *   lam_re[r], lam_im[r]   eigenvalue of each column of Phi_R;
 *   beta[r]                real amplitudes (the coefficient vector at k = 0);
 *   sigma[r]               singular values of the snapshot matrix X (descending);
 *   G[r*q]                 real-form forcing (column-major r x q), DMDc only.
 * A conjugate pair (lambda, conj lambda) with mode phi and amplitude b owns two
 * adjacent columns c, c+1: Phi_R[:, c] = Re phi, Phi_R[:, c+1] = Im phi,
 * lam_im[c] > 0, lam_im[c+1] = -lam_im[c], beta[c] = Re(2b), beta[c+1] = -Im(2b).
 * A real eigenvalue owns one column with lam_im = 0.  Frame k is
 * x_k = Phi_R C[:, k] with, for a pair, y = lambda^k (beta[c] - i beta[c+1]),
 * C[c, k] = Re y, C[c+1, k] = -Im y, and C[c, k] = lambda^k beta[c] for a real
 * column.  Columns are in canonical order: |lambda| descending, then Im
 * descending, each pair's Im > 0 member first.
 */
#ifndef DMD_H
#define DMD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DMD_EXPORT __attribute__((visibility("default")))
#else
#define DMD_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dmd_status;
enum {
  DMD_OK = 0,
  DMD_EINVAL = 1,      /* invalid argument (host check)                         */
  DMD_ENOMEM = 2,      /* workspace smaller than the size query returned        */
  DMD_ENUMERIC = 3,    /* numerical breakdown (Cholesky pivot <= 0, no QR convergence) */
  DMD_ERANK = 4,       /* sigma_r <= 1e-6 sigma_1: requested rank not supported by the data */
  DMD_ENONFINITE = 5,  /* NaN or Inf in the snapshots                            */
  DMD_ETIMEOUT = 6,    /* a bounded device-side wait ran out                    */
  DMD_ECUDA = 7        /* a CUDA runtime call or kernel launch failed            */
};

enum { DMD_FP32 = 0, DMD_MIXED_BF16X3 = 1 };

/* Device status words (int32[DMD_INFO_WORDS]) written by dmd_fit:
 *   info[0] status (dmd_status), info[1] number of conjugate pairs,
 *   info[2] number of real eigenvalues, info[3] QR sweeps used,
 *   info[4] tag of the first failure, info[5] number of sketch directions
 *   dropped by the Gram orthonormalisations (directions the snapshots do not
 *   resolve above rounding). */
#define DMD_INFO_WORDS 8

#define DMD_MODAL_DOUBLES(r, q) ((size_t)(r) * (4 + (size_t)(q)))

/* Fit problem (Sec. 3.1 and Sec. 4.3).  S = [x_0 .. x_m] is n x (m+1) FP32 with
 * leading dimension ldS; X = S[:, 0:m] and X' = S[:, 1:m+1] are views of it.
 * l = min(r + oversample, m) is the sketch width; power_iters the number of
 * power iterations.  q > 0 selects DMD with control (Eq. external_forces):
 * Ups is then q x m FP32 (column k = u_k, leading dimension q).  If Omega is
 * non-NULL it is the m x l FP64 Gaussian test matrix (column-major, ld m);
 * otherwise the library draws it on the device from Philox4x32-10 keyed by
 * `seed`. */
typedef struct dmd_fit_desc {
  int64_t n;
  int64_t ldS;
  int64_t ldPhi;       /* leading dimension of the Phi_R output             */
  int32_t m;
  int32_t r;
  int32_t oversample;
  int32_t power_iters;
  int32_t q;           /* control channels, 0 = plain DMD                    */
  int32_t precision;   /* DMD_FP32 or DMD_MIXED_BF16X3                       */
  uint64_t seed;
} dmd_fit_desc;

/* Frames request for dmd_predict / dmd_predict_backward (Eq. large_time_step).
 * k[0..K) are integer time indices (device int32).  Without control (q == 0)
 * any k is allowed, negative k reverses time (Eq. reverse_simulation).  With
 * control, the reduced state is rolled out z_{t+1} = Lambda z_t + G u_t
 * (Eq. external_forces) for t < steps from z_0 = beta, and every k must lie in
 * [0, steps]; u is q x steps FP32 (column t = u_t, leading dimension q). */
typedef struct dmd_predict_desc {
  int64_t n;
  int64_t ldPhi;
  int64_t ldOut;
  int32_t r;
  int32_t K;
  int32_t q;
  int32_t steps;
  int32_t precision;
  int32_t chunk;       /* frames per recompute chunk of the FP32-form loss (0 = 50) */
} dmd_predict_desc;

/* Per-frame loss of dmd_predict_loss, rho of the residual e = x - target
 * (Sec. 7.2 asks for gradients of the prediction for inverse design and names
 * no loss; the quadratic loss is the plain reading, the Huber loss the
 * general, non-quadratic case). */
typedef enum { DMD_LOSS_QUADRATIC = 0, DMD_LOSS_HUBER = 1 } dmd_loss_kind;
typedef struct dmd_loss_opts {
  int32_t kind;        /* DMD_LOSS_QUADRATIC: rho(e) = e^2 / 2;
                          DMD_LOSS_HUBER: rho(e) = e^2 / 2 for |e| <= delta,
                          delta (|e| - delta / 2) beyond */
  int32_t reserved;    /* 0 */
  double delta;        /* Huber width, > 0 (ignored for the quadratic loss) */
} dmd_loss_opts;

DMD_EXPORT const char* dmd_last_error(void);
DMD_EXPORT const char* dmd_version(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (host-side counter, for accounting in benchmarks). */
DMD_EXPORT uint64_t dmd_launch_count(void);

/* Asynchronous status of the calls that have no info argument (dmd_predict,
 * dmd_predict_backward, dmd_predict_loss, dmd_predict_noalloc,
 * dmd_advect_density and the component kernels): a tensor-core or TMA kernel
 * of such a call whose bounded wait ran out (2 s) writes DMD_ETIMEOUT to
 * words[0] and the site to words[4] of a per-device status word, the first
 * failure winning.  (The fits, dmd_upsample and each scene of
 * dmd_fit_predict_batch report to their own info instead.)
 * Copies the current device's word (DMD_INFO_WORDS int32) into the host
 * array `words` after the work already queued on `stream` has finished
 * (the stream is synchronised), and zeroes it when `clear` is non-zero.
 * The word's device address is looked up once per device, so, as for
 * dmd_predict_noalloc, a device reset (cudaDeviceReset) after the first call
 * of the library on that device is not supported.
 * Errors: DMD_EINVAL for a NULL `words`, DMD_ECUDA if a copy fails. */
DMD_EXPORT dmd_status dmd_async_status(int32_t* words, int32_t clear, void* stream);

/* ---- fit ---------------------------------------------------------------- */

/* Workspace bytes dmd_fit needs for this problem (host-side query, no GPU). */
DMD_EXPORT dmd_status dmd_fit_workspace_bytes(const dmd_fit_desc* desc, size_t* bytes);

/* Fit the exact DMD (or DMDc) model of S.
 * Outputs: Phi_R (n x r FP32, ld desc->ldPhi), modal (DMD_MODAL_DOUBLES(r, q)
 * doubles, layout above), info (DMD_INFO_WORDS int32).  Steps: Philox sketch
 * Omega; Y = X Omega; CholeskyQR2; power iterations; P = Q^T S; SVD of
 * B = P[:, 0:m]; reduced operator A~ = U_B^T (Q^T X') V Sigma^{-1} (Sec. 3.1);
 * eigendecomposition A~ W = W Lambda; modes Phi = X' V Sigma^{-1} W written in
 * real form; amplitudes b = Phi^+ x_0 by least squares in the Q basis
 * (Eq. projection).  Errors: EINVAL if n < 1, m < 2, r < 1, r > min(m, n),
 * r > 512, ldS < n, ldS % 4, ldPhi < n, ldPhi % 4 or a NULL pointer; ENOMEM
 * if ws_bytes is below the query.  The workspace must be 256-byte aligned. */
DMD_EXPORT dmd_status dmd_fit(const dmd_fit_desc* desc, const float* S, const float* Ups,
                   const double* Omega, float* Phi_R, double* modal, int32_t* info,
                   void* workspace, size_t ws_bytes, void* stream);

/* ---- OptDMD (Sec. 4.2, Eqs. variable_projection and phi_optdmd) -------- */

/* Options of dmd_fit_optdmd; zero fields take the defaults. */
typedef struct dmd_optdmd_opts {
  int32_t max_evals;   /* objective evaluations of the Levenberg-Marquardt loop (0 = 40) */
  int32_t reserved;
  double tol;          /* stop when the (taken or predicted) fall of the objective is <= tol of it (0 = 1e-10) */
  double mu0;          /* initial Marquardt damping, relative to diag(J^T J) (0 = 1e-3) */
} dmd_optdmd_opts;

DMD_EXPORT dmd_status dmd_fit_optdmd_workspace_bytes(const dmd_fit_desc* desc, size_t* bytes);

/* OptDMD fit of S (desc->q must be 0).  Runs dmd_fit's randomized SVD
 * X ~ U Sigma V^T (U = Q U_B) and exact-DMD eigenvalues, then fits the
 * eigenvalues alpha over all T = m snapshots at once:
 *   min_{alpha, B} || V Sigma - Phi(alpha) B ||_F,  Phi(alpha)_{t, j} = alpha_j^t (t = 0..T-1),
 * by variable projection (B = Phi^+ V Sigma) and Levenberg-Marquardt on alpha
 * (FP64, conjugate pairs kept, Kaufman's Jacobian, Marquardt damping mu
 * diag(J^T J) with Nielsen's update: a taken step scales mu by
 * max(1/3, 1 - (2 q - 1)^3), q = actual / predicted fall, a refused one by
 * nu = 2, 4, 8, ...), starting from the exact-DMD eigenvalues.  The loop stops
 * when a taken step lowers the objective by at most tol of it or is below
 * 1e-12 of max |p|, when a refused step's predicted fall is at most tol of
 * the objective, when mu exceeds 1e12, or after max_evals evaluations; the
 * decisions are taken on the device (no host synchronisation).  Modes phi_i = U B^T(:, i) / ||U B^T(:, i)||_2 and
 * amplitudes b_i = ||U B^T(:, i)||_2 (so x_t ~ sum_i phi_i b_i alpha_i^t),
 * written in the real form and canonical order of dmd_fit; sigma as dmd_fit.
 * stats (device, 4 doubles, may be NULL): objective at the exact-DMD
 * eigenvalues, final objective, evaluations, accepted steps.  info as
 * dmd_fit (DMD_ENUMERIC if not even the starting point gave a finite
 * objective).  Errors: those of dmd_fit; EINVAL for q > 0 or r > 200. */
DMD_EXPORT dmd_status dmd_fit_optdmd(const dmd_fit_desc* desc, const dmd_optdmd_opts* opts, const float* S,
                          const double* Omega, float* Phi_R, double* modal, int32_t* info,
                          double* stats, void* workspace, size_t ws_bytes, void* stream);

/* ---- upsampling (Sec. 6.3.1) ------------------------------------------- */

/* Upsampling request: a fitted high-resolution model (Phi_R n x r, ld ldPhi;
 * modal of r columns, q = 0) and an input matrix `in` (n x (T+1) FP32, ld ldIn)
 * whose column 0 is the high-resolution initial state H_0 and whose columns
 * 1..T are the inputs L_1..L_T given on the high-resolution grid (e.g. a
 * low-resolution simulation prolonged to it). */
typedef struct dmd_upsample_desc {
  int64_t n;
  int64_t ldPhi;
  int64_t ldIn;
  int64_t ldOut;
  int32_t r;
  int32_t T;
  int32_t precision;
  int32_t gram_given;  /* 1: `gram` holds Phi_R^T Phi_R from an earlier call; 0: compute it (and store it in `gram` if non-NULL) */
  double threshold;    /* low-order modes: |Im log(lambda)| / dt < threshold */
  double dt;           /* time step of the model (> 0)                       */
} dmd_upsample_desc;

DMD_EXPORT dmd_status dmd_upsample_workspace_bytes(const dmd_upsample_desc* desc, size_t* bytes);

/* Upsampling evolution (Sec. 6.3.1): R_0 = Phi^+ H_0 and, for t = 1..T,
 * R_t = S^L Phi^+ L_t + S^H Lambda R_{t-1}, H_t = Phi R_t, where S^L keeps
 * the low-order modes (|Im log(lambda)| / dt < threshold) and S^H the others;
 * Phi^+ is the least-squares projection (G = Phi_R^T Phi_R by a Cholesky
 * factor, Phi_R^T [H_0 | L] by one tall reduction).  G depends on the model
 * only: `gram` (device, r x r FP64, may be NULL) receives it, and a later
 * call with gram_given = 1 reuses it instead of the pass over Phi_R.  Lambda being diagonal,
 * the high-order part is Lambda^t R_0 in closed form, so all T frames are one
 * tall product out = Phi_R C (out: n x T FP32, ld ldOut, column t-1 = H_t).
 * info (DMD_INFO_WORDS int32, device): DMD_ENUMERIC if G is not positive
 * definite; modes that are numerically dependent are dropped (info[5]).
 * Errors: EINVAL for bad sizes (n < 1, r < 1, r > 200, T < 1, ld* < n or not
 * a multiple of 4, dt <= 0, threshold < 0), NULL pointers or gram_given
 * without gram; ENOMEM if
 * ws_bytes is below the query. */
DMD_EXPORT dmd_status dmd_upsample(const dmd_upsample_desc* desc, const float* Phi_R, const double* modal,
                        const float* in, float* out, double* gram, int32_t* info, void* workspace,
                        size_t ws_bytes, void* stream);

/* ---- density in the DMD velocity (Sec. 7.2) ----------------------------- */

/* A model of velocity snapshots on a periodic N^dim MAC grid (dim 2 or 3,
 * n = dim N^dim: component d of a frame on the low d-face of each cell, cells
 * in C order over the axes) and a cell-centred density (N^dim FP32). */
typedef struct dmd_advect_desc {
  int64_t ldPhi;
  int64_t ldRho;       /* leading dimension of the density frames (>= N^dim, multiple of 4) */
  int32_t N;
  int32_t dim;
  int32_t r;
  int32_t K;           /* steps: velocity frames u_0 .. u_{K-1}                  */
  int32_t precision;
  int32_t chunk;       /* velocity frames reconstructed per batch (0 = 256)       */
  double dt;           /* step in grid cells per unit velocity                    */
} dmd_advect_desc;

DMD_EXPORT dmd_status dmd_advect_workspace_bytes(const dmd_advect_desc* desc, size_t* bytes);

/* Density advected by the model's velocity (Sec. 7.2: velocity from the DMD
 * model, density by classical integration in it): rho_{k+1}(c) =
 * rho_k(c - dt u_k(c)), u_k = x_k of the model (Eq. large_time_step) at the
 * centre of cell c (mean of the two faces per axis), rho_k by multilinear
 * interpolation with periodic wrap.  rho (N^dim x (K+1) FP32, ld ldRho)
 * receives rho_0 = rho0 and rho_1 .. rho_K.  Velocity frames are rebuilt in
 * batches of `chunk` by the reconstruction product.  Errors: EINVAL for bad
 * sizes (dim not 2 or 3, N < 2, N above 32768 (2D) or 1024 (3D), r < 1, K < 1, ldPhi < dim N^dim, ldRho <
 * N^dim, leading dimensions not multiples of 4, non-finite dt) or NULL
 * pointers; ENOMEM if ws_bytes is below the query. */
DMD_EXPORT dmd_status dmd_advect_density(const dmd_advect_desc* desc, const float* Phi_R, const double* modal,
                              const float* rho0, float* rho, void* workspace, size_t ws_bytes,
                              void* stream);

/* ---- prediction (Eq. large_time_step, Eq. reverse_simulation, Eq. external_forces) */

/* Workspace bytes of dmd_predict and dmd_predict_backward (host-side query). */
DMD_EXPORT dmd_status dmd_predict_workspace_bytes(const dmd_predict_desc* desc, size_t* bytes);

/* out (n x K FP32, ld desc->ldOut): frame j is x_{k[j]} = Phi_R C[:, j].
 * The coefficients C are formed in FP64 on the device (lambda^k in polar form:
 * |lambda|^k = exp(k log|lambda|), angle k*arg(lambda)); the reconstruction is
 * one real GEMM Phi_R * C in the requested precision. */
DMD_EXPORT dmd_status dmd_predict(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                       const int32_t* k, const float* u, float* out,
                       void* workspace, size_t ws_bytes, void* stream);

/* Adjoint of dmd_predict.  dOut (n x K FP32, ld desc->ldOut) is dL/d(out).
 * Writes d_modal (same layout as modal: dL/dRe(lambda), dL/dIm(lambda) per
 * column -- a pair's value is stored in both its columns and belongs to the
 * Im > 0 member --, dL/dbeta, zero for sigma, dL/dG for DMDc) and, with
 * control, d_u (q x steps FP32) = dL/du_t.  Steps: dC = Phi_R^T dOut (split
 * over n, FP64 reduction), then the FP64 chain rule through lambda^k and the
 * reverse recursion mu_t = L^T mu_{t+1} + dC_t of the rollout. */
DMD_EXPORT dmd_status dmd_predict_backward(const dmd_predict_desc* desc, const float* Phi_R,
                                const double* modal, const int32_t* k, const float* u,
                                const float* dOut, double* d_modal, float* d_u,
                                void* workspace, size_t ws_bytes, void* stream);

/* Streamed per-frame loss L = sum_j w_j sum_i rho(x_{k[j]},i - target_i)
 * (rho of dmd_loss_opts; opts NULL = quadratic, L = sum_j w_j ||x - target||^2 / 2)
 * without storing the trajectory.  target: n FP32; w: K FP64 weights
 * (device).  loss: one double (device).  With want_grad != 0 the gradient
 * dC = Phi_R^T G, G_ij = w_j rho'(x_ij - target_i), is taken and d_modal /
 * d_u are written as dmd_predict_backward does.
 * Mixed form (r <= 160): the frames never reach memory.  The loss alone is
 * the reconstruction kernel with a loss epilogue (Phi_R read once); with the
 * gradient Phi_R is first copied once into the workspace as bf16 hi / lo
 * planes in the tensor cores' operand layout (4 bytes per row and mode,
 * r padded to a multiple of 16), then one kernel recomputes each 128-row x
 * 128-frame tile on the tensor cores from that copy, forms G in its
 * epilogue, keeps G in tensor memory and accumulates dC^T += G^T Phi_tile
 * there (the copy read once per 128 frames), with FP64 partials per CTA
 * summed in a fixed order.
 * FP32 form (and r > 160): frames are recomputed in chunks of desc->chunk;
 * each chunk is written, turned into G by a loss kernel and reduced by the
 * Phi_R^T G pass. */
DMD_EXPORT dmd_status dmd_predict_loss_workspace_bytes(const dmd_predict_desc* desc, int32_t want_grad,
                                                       size_t* bytes);
DMD_EXPORT dmd_status dmd_predict_loss(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                            const int32_t* k, const float* u, const float* target,
                            const double* w, const dmd_loss_opts* opts, int32_t want_grad, double* loss,
                            double* d_modal, float* d_u, void* workspace, size_t ws_bytes,
                            void* stream);

/* ---- prediction without allocation --------------------------------------- */

/* Size of the library's fixed device scratch array used by dmd_predict_noalloc
 * (held on every GPU that loads the library until the process exits). */
#define DMD_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)

/* dmd_predict for callers that cannot allocate GPU memory.  The paper has no
 * counterpart: it is an interface for applications that drive the prediction
 * from an interactive frame loop, reserve their GPU memory once under their
 * own allocator and forbid cudaMalloc / cudaFree afterwards (those calls can
 * synchronise the device and stall a frame), or that host this library as a
 * plug-in without giving it an allocator.
 * Arguments, layouts and results are those of dmd_predict: the caller owns
 * and passes every input and the output frames; the workspace comes from a
 * fixed DMD_NOALLOC_SCRATCH_BYTES array inside the library instead.  Nothing
 * is allocated: no cudaMalloc, no cudaFree, no allocating library routine.
 * Limits and errors: DMD_EINVAL (with a message naming the bytes needed) when
 * the forward pass's workspace (the r x K FP64 coefficients, the control
 * rollout and the product's scratch) exceeds DMD_NOALLOC_SCRATCH_BYTES; for
 * r = 150 without control that is about K = 9000 frames.  Otherwise the
 * errors of dmd_predict.
 * Set-up: the first call on each device looks up the array's device address
 * on that (current) device; make that first call before any stream capture.
 * The address is kept for the life of the process: a device reset
 * (cudaDeviceReset) after the first call is not supported.
 * Sharing: every call on a device uses the same array, and the array keeps
 * the previous call's contents (each call clears the part it uses before
 * use).  Calls whose GPU work overlaps -- on different streams, or from
 * different host threads -- race on the array and give wrong frames; order
 * them on one stream or with events. */
DMD_EXPORT dmd_status dmd_predict_noalloc(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                               const int32_t* k, const float* u, float* out, void* stream);

/* Temporal editing of a fitted model (Eq. edit_temporal): with
 * Omega = log(lambda) / dt, every mode with |Im Omega| < threshold belongs to
 * the low-frequency cluster (the paper uses 0.01), the others to the
 * high-frequency cluster; each cluster's edit {w, s_re, s_im} (host arrays of
 * 3 doubles: low, high) gives lambda' = exp((s_re Re Omega + i s_im Im Omega) dt)
 * and beta' = w beta (the mode's weight).  Conjugate partners get conjugate
 * edits; a negative real eigenvalue keeps its sign.  modal_out (a separate
 * DMD_MODAL_DOUBLES(r, q) buffer) then feeds dmd_predict like a fitted model;
 * sigma and G are copied.  Errors: EINVAL for bad sizes, dt <= 0, negative
 * threshold or aliasing buffers. */
DMD_EXPORT dmd_status dmd_edit_modes(int32_t r, int32_t q, const double* modal_in, double* modal_out,
                          double threshold, const double* low, const double* high, double dt, void* stream);

/* Autotuner of the reconstruction (no counterpart in the paper: it picks the
 * tensor-core tile configuration of Phi_R C for this GPU).  With the
 * operands of a dmd_predict call (desc->q must be 0; mixed precision; K > 256
 * frames), every (frame-chunk width, A stages, B ring entries) configuration that
 * fits in shared memory is launched and timed with CUDA events on `stream`,
 * and the fastest is kept for all later predictions with the same number of
 * modes (per process).  chosen (3 int32, may be NULL) receives (chunk width,
 * A stages, B ring entries), zeros when nothing was tuned.  `out` is overwritten
 * with the frames.  Synchronises `stream`: call it before any capture. */
DMD_EXPORT dmd_status dmd_autotune_predict(const dmd_predict_desc* desc, const float* Phi_R, const double* modal,
                                const int32_t* k, float* out, void* workspace, size_t ws_bytes,
                                void* stream, int32_t* chosen);

/* ---- many scenes at once ----------------------------------------------- */

/* One scene of a batch: its fit (no control inputs: fit.q must be 0) and,
 * with K > 0, the prediction of K frames k[0..K) into out (n x K FP32,
 * ld ldOut).  Pointers are device pointers owned by the caller. */
typedef struct dmd_scene {
  dmd_fit_desc fit;
  const float* S;       /* (m+1) snapshots, n x (m+1), ld fit.ldS           */
  float* Phi_R;         /* n x r, ld fit.ldPhi                               */
  double* modal;        /* DMD_MODAL_DOUBLES(r, 0)                           */
  int32_t* info;        /* DMD_INFO_WORDS                                    */
  int32_t K;            /* frames to predict (0: fit only)                   */
  const int32_t* k;     /* K time indices                                    */
  float* out;           /* n x K frames, ld ldOut                            */
  int64_t ldOut;
} dmd_scene;

/* Workspace bytes of dmd_fit_predict_batch for these scenes and lanes. */
DMD_EXPORT dmd_status dmd_batch_workspace_bytes(int32_t count, const dmd_scene* scenes, int32_t lanes,
                                     size_t* bytes);

/* Fit (Sec. 3.1, Sec. 4.3) and predict (Eq. large_time_step) `count`
 * independent scenes of any sizes.  The scenes run concurrently on `lanes`
 * internal streams (0 = 16, at most 32), assigned longest first (by n (m+1))
 * to the least-loaded lane; each lane reuses one slice of the workspace,
 * sized for its largest scene.  The lanes fork from and join back into
 * `stream` through events, so the whole batch is ordered on `stream` and, when
 * `stream` is being captured, is captured (a batch then replays as one graph
 * launch).  Every scene's results equal those of dmd_fit + dmd_predict on the
 * same inputs.  The first call on a device creates the lanes: make it before
 * any capture.  Calls on one device share the lanes: do not overlap them.
 * Errors: EINVAL for a bad scene (NULL pointers, q > 0, bad ldOut) or any
 * argument error of dmd_fit; ENOMEM if ws_bytes is below the query. */
DMD_EXPORT dmd_status dmd_fit_predict_batch(int32_t count, const dmd_scene* scenes, int32_t lanes,
                                 void* workspace, size_t ws_bytes, void* stream);

/* ---- component entry points (the building blocks, exposed for tests) ------ */

/* Omega (m x l FP64, ld m) ~ N(0, 1) from Philox4x32-10 (Salmon et al. 2011):
 * element e uses counter (e/4 lo, e/4 hi, 0x0D3D0001, 0), key (seed lo, seed hi)
 * and output e % 4 of two Box-Muller pairs.  The randomized range finder of
 * Sec. 4.3 multiplies X by this matrix. */
DMD_EXPORT dmd_status dmd_sketch_matrix(int32_t m, int32_t l, uint64_t seed, double* Omega, void* stream);

/* Raw Philox4x32-10 blocks: out[4*i .. 4*i+3] = philox(ctr = (i lo, i hi, stream_id, 0), key). */
DMD_EXPORT dmd_status dmd_philox_blocks(int64_t count, uint32_t stream_id, uint64_t key, uint32_t* out,
                             void* stream);

/* Tall product C = A * B (the sketch X*Omega, the power step X*Z, the modes
 * X'*M of Sec. 4.3 / Sec. 3.1 and the reconstruction Phi_R*C of
 * Eq. large_time_step).  A: n x Kd FP32 (lda); B: Kd x N FP64 (ld Kd),
 * rounded to FP32 or split to bf16 hi/lo inside; C: n x N FP32 (ldc).
 * If gram != NULL it also writes the N x N FP64 Gram C^T C of the FP32 result. */
DMD_EXPORT dmd_status dmd_gemm_tall_workspace_bytes(int32_t precision, int64_t n, int32_t Kd, int32_t N,
                                         size_t* bytes);
DMD_EXPORT dmd_status dmd_gemm_tall(int32_t precision, int64_t n, int32_t Kd, int32_t N, const float* A,
                         int64_t lda, const double* B, float* C, int64_t ldc, double* gram,
                         void* workspace, size_t ws_bytes, void* stream);

/* Reduction over the tall dimension C = A^T B (the power step X^T Q, the
 * projection Q^T S of Sec. 4.3 and Gram matrices).  A: n x Ka FP32 (lda),
 * B: n x N FP32 (ldb), C: Ka x N FP64 (ld Ka).  Per-block partial sums are
 * FP64 and are added in a fixed order, so the result is bitwise reproducible. */
DMD_EXPORT dmd_status dmd_gemm_tn_workspace_bytes(int32_t precision, int64_t n, int32_t Ka, int32_t N,
                                       size_t* bytes);
DMD_EXPORT dmd_status dmd_gemm_tn(int32_t precision, int64_t n, int32_t Ka, int32_t N, const float* A,
                       int64_t lda, const float* B, int64_t ldb, double* C,
                       void* workspace, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DMD_H */
