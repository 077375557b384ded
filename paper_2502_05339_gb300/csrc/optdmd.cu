// OptDMD (Sec. 4.2, Eqs. variable_projection and phi_optdmd) on the device.
//
// Given the rank-r SVD X ~ U Sigma V^T of the snapshots x_0 .. x_{T-1}
// (T = m; here the randomized one of the fit, U = Q U_B with Q = Q1 T2) and the
// exact-DMD eigenvalues as the starting point, fit alpha in
//     min_{alpha, B} || V Sigma - Phi(alpha) B ||_F,   Phi(alpha)_{t, j} = alpha_j^t,
// by variable projection: for fixed alpha the best B is Phi^+ Y (Y = V Sigma),
// and Levenberg-Marquardt runs on the projected residual rho = (I - P) Y,
// P = Phi Phi^+.  Then phi_i = U B^T(:, i) / ||U B^T(:, i)||_2 with amplitude
// b_i = ||U B^T(:, i)||_2, lifted by one tall product Q1 M.
//
// Real 2x2 form.  Real snapshots keep the eigenvalues closed under
// conjugation, so the unknowns are r reals p: (Re alpha, Im alpha) of each
// pair's first member and each real eigenvalue; the basis is real, a pair
// owning the columns Re alpha^t and Im alpha^t (the span of alpha^t and
// conj(alpha)^t).  With d_t = t alpha^(t-1) stored as derivative columns D
// (Re d, Im d), d Phi / d Re alpha = (Re d, Im d) and
// d Phi / d Im alpha = (-Im d, Re d) in the pair's two columns.
//
// Jacobian (Kaufman's form): column k is -(I - P) (d Phi / d p_k) B, a sum of
// at most two outer products e_j b_i^T with e_j a column of E = (I - P) D and
// b_i a row of B, so
//     (J^T J)_{kl} = sum s s' (E^T E)_{j j'} (B B^T)_{i i'},
//     (J^T rho)_k  = -sum s (E^T rho B^T)_{j i},
// r x r products only.  The projection is taken from the normal equations
// G = Phi^T Phi = R^T R (FP64 Cholesky; R^{-1} by columns, then products)
// with one refinement step.
//
// Control flow stays on the device: a decision kernel accepts the trial point
// when the objective falls or rejects it (Levenberg-Marquardt damping with
// Nielsen's update, see k_opt_decide), and sets a stop
// flag on convergence; every later kernel of the loop then returns at once.
// A fixed number of evaluations is therefore launched with no host
// synchronisation, and the whole fit can be captured in a CUDA graph.
#include <float.h>

#include "optdmd.cuh"

namespace dmd {

dmd_status dgemm_gated(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B,
                       int ldb, bool tb, double beta, double* C, int ldc, const int32_t* skip, cudaStream_t st);
dmd_status cholesky_upper_gated(int n, double* G, int ld, double tau, int32_t* info, int tag, const int32_t* skip,
                                cudaStream_t st);
dmd_status dgemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B, int ldb,
                 bool tb, double beta, double* C, int ldc, cudaStream_t st);
dmd_status chol_solve_gated(int n, const double* R, int ldr, const double* Bm, int ldb, int ncols, double alpha,
                            double beta, double* X, int ldx, const int32_t* skip, cudaStream_t st);
dmd_status tri_inv_upper_gated(int n, const double* R, int ldr, double* T, int ldt, const int32_t* skip,
                               cudaStream_t st);

namespace {

// state words: doubles sd[] and ints si[]
enum { SD_F = 0, SD_MU, SD_F0, SD_EVALS, SD_ACCEPTED, SD_NU, SD_WORDS };
enum { SI_DONE = 0, SI_FIRST, SI_WORDS };

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// a^k, k >= 0, by repeated squaring (about 2 log2 k products).
__device__ double2 cpow_int(double2 a, int k) {
  double2 r = make_double2(1.0, 0.0);
  while (k) {
    if (k & 1) r = cmul(r, a);
    a = cmul(a, a);
    k >>= 1;
  }
  return r;
}

// Column kinds from the exact fit's layout (pairs adjacent, Im > 0 first):
// 1 = pair (Re, Im), 2 = its second column, 0 = real.  Starting parameters
// and solver state.
__global__ void k_opt_init(int r, const double* __restrict__ modal, int* __restrict__ kinds,
                           double* __restrict__ pt, double* __restrict__ sd, int32_t* __restrict__ si, double mu0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double* lre = modal;
  const double* lim = modal + r;
  int c = 0;
  while (c < r) {
    if (lim[c] > 0.0 && c + 1 < r) {
      kinds[c] = 1;
      kinds[c + 1] = 2;
      pt[c] = lre[c];
      pt[c + 1] = lim[c];
      c += 2;
    } else {
      kinds[c] = 0;
      pt[c] = lre[c];
      c += 1;
    }
  }
  sd[SD_F] = DBL_MAX;
  sd[SD_MU] = mu0;
  sd[SD_F0] = 0.0;
  sd[SD_EVALS] = 0.0;
  sd[SD_ACCEPTED] = 0.0;
  sd[SD_NU] = 2.0;
  si[SI_DONE] = 0;
  si[SI_FIRST] = 1;
}

// Phi (T x r) and D (T x r) at the trial parameters: column pair (c, c+1)
// = (Re z, Im z), z = alpha^t, and (Re d, Im d), d = t alpha^(t-1); a real
// column a^t and t a^(t-1).
__global__ void k_opt_basis(int T, int r, const int* __restrict__ kinds, const double* __restrict__ pt,
                            double* __restrict__ Phi, int ldp, double* __restrict__ D, int ldd,
                            const int32_t* __restrict__ skip) {
  if (*skip) return;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)T * r) return;
  const int t = (int)(idx % T), c = (int)(idx / T);
  const int kind = kinds[c];
  if (kind == 2) return;
  const double2 a = make_double2(pt[c], kind == 1 ? pt[c + 1] : 0.0);
  double2 z = make_double2(1.0, 0.0), d = make_double2(0.0, 0.0);
  if (t > 0) {
    const double2 w = cpow_int(a, t - 1);
    z = cmul(w, a);
    d = make_double2(t * w.x, t * w.y);
  }
  Phi[t + (int64_t)c * ldp] = z.x;
  D[t + (int64_t)c * ldd] = d.x;
  if (kind == 1) {
    Phi[t + (int64_t)(c + 1) * ldp] = z.y;
    D[t + (int64_t)(c + 1) * ldd] = d.y;
  }
}

// Terms (j, i, s) of parameter k: d Phi / d p_k B = sum s D_j b_i^T.
__device__ __forceinline__ int param_terms(const int* kinds, int k, int* j, int* i, double* s) {
  const int kind = kinds[k];
  if (kind == 0) {
    j[0] = k; i[0] = k; s[0] = 1.0;
    return 1;
  }
  if (kind == 1) {   // Re alpha: (Re d, Im d) in columns (k, k+1)
    j[0] = k; i[0] = k; s[0] = 1.0;
    j[1] = k + 1; i[1] = k + 1; s[1] = 1.0;
    return 2;
  }
  // Im alpha of the pair (k-1, k): (-Im d, Re d) in columns (k-1, k)
  j[0] = k; i[0] = k - 1; s[0] = -1.0;
  j[1] = k - 1; i[1] = k; s[1] = 1.0;
  return 2;
}

// J^T J and J^T rho of the trial point from Ge = E^T E, Gb = B B^T and
// Hh = E^T rho B^T (all r x r, ld r).
__global__ void k_opt_assemble(int r, const int* __restrict__ kinds, const double* __restrict__ Ge,
                               const double* __restrict__ Gb, const double* __restrict__ Hh,
                               double* __restrict__ JtJ, double* __restrict__ g, const int32_t* __restrict__ skip) {
  if (*skip) return;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)r * r) return;
  const int k = (int)(idx % r), l = (int)(idx / r);
  int jk[2], ik[2], jl[2], il[2];
  double sk[2], sl[2];
  const int nk = param_terms(kinds, k, jk, ik, sk);
  const int nl = param_terms(kinds, l, jl, il, sl);
  double acc = 0.0;
  for (int a = 0; a < nk; ++a)
    for (int b = 0; b < nl; ++b)
      acc = fma(sk[a] * sl[b] * Ge[jk[a] + (int64_t)jl[b] * r], Gb[ik[a] + (int64_t)il[b] * r], acc);
  JtJ[k + (int64_t)l * r] = acc;
  if (l == 0) {
    double gk = 0.0;
    for (int a = 0; a < nk; ++a) gk = fma(-sk[a], Hh[jk[a] + (int64_t)ik[a] * r], gk);
    g[k] = gk;
  }
}

// Accept / reject the trial point and prepare the next step's system
// A = J^T J + mu diag(J^T J) (of the kept point) and the step's base point.
// The linear model's predicted fall of f = ||rho||^2 for the step
// delta = pt - p is pred = -(2 g.delta + delta.J^T J.delta); a taken step
// scales mu by max(1/3, 1 - (2 q - 1)^3), q = actual / predicted fall, and
// resets nu = 2; a refused one multiplies mu by nu and doubles nu (Nielsen's
// update).  One CTA.  rho = RE[:, 0:r] (T x r, ld T); Bt = B of the trial
// (r x r, ld r).
__global__ void __launch_bounds__(512) k_opt_decide(int T, int r, const double* __restrict__ RE,
                                                    double* __restrict__ pt, double* __restrict__ p,
                                                    const double* __restrict__ JtJt, const double* __restrict__ gt,
                                                    double* __restrict__ JtJ, double* __restrict__ g,
                                                    const double* __restrict__ Bt, double* __restrict__ Bk,
                                                    double* __restrict__ A, double* __restrict__ sd,
                                                    int32_t* __restrict__ si, double tol) {
  __shared__ double red[32];
  if (si[SI_DONE]) return;
  const int tid = threadIdx.x, bd = blockDim.x;
  double loc = 0.0;
  const int64_t cnt = (int64_t)T * r;
  for (int64_t e = tid; e < cnt; e += bd) loc = fma(RE[e], RE[e], loc);
  const double ft = block_sum(loc, red);
  double dstep = 0.0, pmax = 0.0;
  for (int i = tid; i < r; i += bd) {
    dstep = fmax(dstep, fabs(pt[i] - p[i]));
    pmax = fmax(pmax, fabs(pt[i]));
  }
  dstep = block_max(dstep, red);
  pmax = block_max(pmax, red);
  const bool first = si[SI_FIRST] != 0;
  double lin = 0.0, quad = 0.0;
  if (!first) {
    const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    for (int a = warp; a < r; a += nw) {
      double acc = 0.0;
      for (int b = lane; b < r; b += 32) acc = fma(JtJ[b + (int64_t)a * r], pt[b] - p[b], acc);
      acc = warp_sum(acc);
      if (lane == 0) quad = fma(pt[a] - p[a], acc, quad);
    }
    for (int i = tid; i < r; i += bd) lin = fma(g[i], pt[i] - p[i], lin);
  }
  lin = block_sum(lin, red);
  quad = block_sum(quad, red);
  const double pred = -(2.0 * lin + quad);
  const double f = sd[SD_F], mu = sd[SD_MU], nu = sd[SD_NU];
  const bool accept = first ? (bool)isfinite(ft) : (ft < f);
  double newmu, newnu;
  bool stop;
  if (accept) {
    if (first) {
      newmu = mu;
      newnu = nu;
      stop = false;
    } else {
      const double q = pred > 0.0 ? (f - ft) / pred : 0.5;
      const double c = 2.0 * q - 1.0;
      newmu = mu * fmax(1.0 / 3.0, 1.0 - c * c * c);
      newnu = 2.0;
      stop = (f - ft) <= tol * f || dstep <= 1e-12 * fmax(1.0, pmax);
    }
  } else {
    newmu = mu * nu;
    newnu = 2.0 * nu;
    stop = first || pred <= tol * f || newmu > 1e12;   // a non-finite start cannot be improved on
  }
  __syncthreads();   // every thread has read the state before it changes
  const int64_t rr = (int64_t)r * r;
  const double* Jsrc = accept ? JtJt : JtJ;
  for (int64_t e = tid; e < rr; e += bd) {
    const double v = Jsrc[e];
    const int a = (int)(e % r), b = (int)(e / r);
    A[e] = (a == b) ? fma(newmu, v, v) : v;
    if (accept) {
      JtJ[e] = v;
      Bk[e] = Bt[e];
    }
  }
  for (int i = tid; i < r; i += bd) {
    if (accept) {
      p[i] = pt[i];
      g[i] = gt[i];
    } else {
      pt[i] = p[i];
    }
  }
  if (tid == 0) {
    if (accept) {
      sd[SD_F] = ft;
      if (first) sd[SD_F0] = ft;
      else sd[SD_ACCEPTED] += 1.0;
      si[SI_FIRST] = 0;
    }
    sd[SD_MU] = newmu;
    sd[SD_NU] = newnu;
    sd[SD_EVALS] += 1.0;
    if (stop) si[SI_DONE] = 1;
  }
}

// Final model in the canonical order (|lambda| descending, then Im
// descending, pairs adjacent with Im > 0 first): eigenvalues, amplitudes
// b = ||U B^T(:, i)|| (= the norm of B's rows for orthonormal U) and the
// small factor Wt (r x r) of the modes, Phi_R = U Bk^T Wt-columns:
// Wt[:, o] = B row / ||w|| with the pair's second row negated (Im phi), and
// sign-flipped again when the fitted Im alpha is negative (the conjugate is
// taken as the pair's first member).
__global__ void __launch_bounds__(256) k_opt_layout(int r, const int* __restrict__ kinds, const double* __restrict__ p,
                                                    const double* __restrict__ Bk, double* __restrict__ modal,
                                                    double* __restrict__ Wt, int32_t* __restrict__ info,
                                                    const double* __restrict__ sd, double* __restrict__ stats) {
  const int tid = threadIdx.x, bd = blockDim.x;
  if (tid == 0) {
    if (!isfinite(sd[SD_F]) || sd[SD_F] == DBL_MAX) raise_status(info, DMD_ENUMERIC, 8100);
    if (stats) {
      stats[0] = sd[SD_F0];
      stats[1] = sd[SD_F];
      stats[2] = sd[SD_EVALS];
      stats[3] = sd[SD_ACCEPTED];
    }
  }
  for (int h = tid; h < r; h += bd) {
    const int kind = kinds[h];
    if (kind == 2) continue;
    const double im = kind == 1 ? fabs(p[h + 1]) : 0.0;
    const double mod = hypot(p[h], im);
    int pos = 0;
    for (int q = 0; q < r; ++q) {
      const int kq = kinds[q];
      if (kq == 2 || q == h) continue;
      const double imq = kq == 1 ? fabs(p[q + 1]) : 0.0;
      const double modq = hypot(p[q], imq);
      const bool before = modq > mod || (modq == mod && (imq > im || (imq == im && q < h)));
      if (before) pos += (kq == 1) ? 2 : 1;
    }
    double nrm = 0.0;
    for (int x = 0; x < r; ++x) {
      const double u = Bk[h + (int64_t)x * r];
      nrm = fma(u, u, nrm);
      if (kind == 1) {
        const double v = Bk[h + 1 + (int64_t)x * r];
        nrm = fma(v, v, nrm);
      }
    }
    nrm = sqrt(nrm);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    const int o = pos;
    modal[o] = p[h];
    modal[r + o] = im;
    modal[2 * r + o] = nrm;
    for (int x = 0; x < r; ++x) Wt[x + (int64_t)o * r] = Bk[h + (int64_t)x * r] * inv;
    if (kind == 1) {
      const double sg = p[h + 1] >= 0.0 ? 1.0 : -1.0;
      modal[o + 1] = p[h];
      modal[r + o + 1] = -im;
      modal[2 * r + o + 1] = 0.0;
      for (int x = 0; x < r; ++x) Wt[x + (int64_t)(o + 1) * r] = -sg * Bk[h + 1 + (int64_t)x * r] * inv;
    }
  }
}

}  // namespace

void carve_optdmd(Arena& a, int T, int r, int l, OptBufs& o) {
  const size_t Tr = (size_t)T * r, rr = (size_t)r * r;
  o.YD = a.take<double>(2 * Tr);
  o.Phi = a.take<double>(Tr);
  o.RE = a.take<double>(2 * Tr);
  o.G = a.take<double>(rr);
  o.Ri = a.take<double>(rr);
  o.H2 = a.take<double>(2 * rr);
  o.H = a.take<double>(2 * rr);
  o.BC = a.take<double>(2 * rr);
  o.EtRE = a.take<double>(2 * rr);
  o.Gb = a.take<double>(rr);
  o.Hh = a.take<double>(rr);
  o.JtJt = a.take<double>(rr);
  o.gt = a.take<double>(r);
  o.JtJ = a.take<double>(rr);
  o.g = a.take<double>(r);
  o.Bk = a.take<double>(rr);
  o.A = a.take<double>(rr);
  o.p = a.take<double>(r);
  o.pt = a.take<double>(r);
  o.sd = a.take<double>(SD_WORDS);
  o.Z = a.take<double>((size_t)l * r);
  o.Wt = a.take<double>(rr);
  o.Mlift = a.take<double>((size_t)l * r);
  o.kinds = a.take<int>(r);
  o.si = a.take<int32_t>(SI_WORDS);
  o.sinfo = a.take<int32_t>(DMD_INFO_WORDS);
}

dmd_status optdmd_small(int T, int r, int l, const double* Bsnap, const double* UB, const double* T2, double* modal,
                        int32_t* info, double* stats, const dmd_optdmd_opts& opt, OptBufs& o, cudaStream_t st) {
  const int max_evals = opt.max_evals > 0 ? opt.max_evals : 40;
  const double tol = opt.tol > 0.0 ? opt.tol : 1e-10;
  const double mu0 = opt.mu0 > 0.0 ? opt.mu0 : 1e-3;
  const size_t Tr = (size_t)T * r;
  const int32_t* skip = o.si + SI_DONE;
  DMD_CUDA_TRY(cudaMemsetAsync(o.sinfo, 0, DMD_INFO_WORDS * sizeof(int32_t), st));
  DMD_CUDA_TRY(cudaMemsetAsync(o.p, 0, (size_t)r * sizeof(double), st));
  k_opt_init<<<1, 32, 0, st>>>(r, modal, o.kinds, o.pt, o.sd, o.si, mu0);
  DMD_LAUNCH_CHECK();
  // Y = V Sigma = B^T U_r (T x r) in the first r columns of [Y | D]
  DMD_TRY(dgemm(T, r, l, 1.0, Bsnap, l, true, UB, l, false, 0.0, o.YD, T, st));
  double* D = o.YD + Tr;
  double* E = o.RE + Tr;
  const unsigned nb_basis = (unsigned)ceil_div((int64_t)T * r, 256);
  const unsigned nb_rr = (unsigned)ceil_div((int64_t)r * r, 256);
  for (int it = 0; it < max_evals; ++it) {
    k_opt_basis<<<nb_basis, 256, 0, st>>>(T, r, o.kinds, o.pt, o.Phi, T, D, T, skip);
    DMD_LAUNCH_CHECK();
    // projection by the normal equations G = Phi^T Phi = R^T R, one refinement step
    DMD_TRY(dgemm_gated(r, r, T, 1.0, o.Phi, T, true, o.Phi, T, false, 0.0, o.G, r, skip, st));
    DMD_TRY(cholesky_upper_gated(r, o.G, r, 1e-14, o.sinfo, 81, skip, st));
    DMD_TRY(tri_inv_upper_gated(r, o.G, r, o.Ri, r, skip, st));
    for (int pass = 0; pass < 2; ++pass) {
      // [B | C] (+)= R^{-1} R^{-T} Phi^T [Y | D]  (pass 0), ... Phi^T [rho | E]  (pass 1)
      DMD_TRY(dgemm_gated(r, 2 * r, T, 1.0, o.Phi, T, true, pass == 0 ? o.YD : o.RE, T, false, 0.0, o.H, r, skip,
                          st));
      DMD_TRY(dgemm_gated(r, 2 * r, r, 1.0, o.Ri, r, true, o.H, r, false, 0.0, o.H2, r, skip, st));
      DMD_TRY(dgemm_gated(r, 2 * r, r, 1.0, o.Ri, r, false, o.H2, r, false, pass == 0 ? 0.0 : 1.0, o.BC, r, skip,
                          st));
      DMD_CUDA_TRY(cudaMemcpyAsync(o.RE, o.YD, 2 * Tr * sizeof(double), cudaMemcpyDeviceToDevice, st));
      DMD_TRY(dgemm_gated(T, 2 * r, r, -1.0, o.Phi, T, false, o.BC, r, false, 1.0, o.RE, T, skip, st));
    }
    // [E^T rho | E^T E], B B^T, E^T rho B^T  ->  J^T J, J^T rho
    DMD_TRY(dgemm_gated(r, 2 * r, T, 1.0, E, T, true, o.RE, T, false, 0.0, o.EtRE, r, skip, st));
    DMD_TRY(dgemm_gated(r, r, r, 1.0, o.BC, r, false, o.BC, r, true, 0.0, o.Gb, r, skip, st));
    DMD_TRY(dgemm_gated(r, r, r, 1.0, o.EtRE, r, false, o.BC, r, true, 0.0, o.Hh, r, skip, st));
    k_opt_assemble<<<nb_rr, 256, 0, st>>>(r, o.kinds, o.EtRE + (size_t)r * r, o.Gb, o.Hh, o.JtJt, o.gt, skip);
    DMD_LAUNCH_CHECK();
    k_opt_decide<<<1, 512, 0, st>>>(T, r, o.RE, o.pt, o.p, o.JtJt, o.gt, o.JtJ, o.g, o.BC, o.Bk, o.A, o.sd, o.si,
                                    tol);
    DMD_LAUNCH_CHECK();
    if (it + 1 == max_evals) break;   // the last evaluation is only accepted or refused
    // step: (J^T J + mu diag) delta = -J^T rho, pt = p + delta
    DMD_TRY(cholesky_upper_gated(r, o.A, r, 1e-15, o.sinfo, 82, skip, st));
    DMD_TRY(chol_solve_gated(r, o.A, r, o.g, r, 1, -1.0, 1.0, o.pt, r, skip, st));
  }
  k_opt_layout<<<1, 256, 0, st>>>(r, o.kinds, o.p, o.Bk, modal, o.Wt, info, o.sd, stats);
  DMD_LAUNCH_CHECK();
  // U_r = Q1 (T2 U_B,r); modes' factor Mlift = T2 U_B,r Wt
  DMD_TRY(dgemm(l, r, l, 1.0, T2, l, false, UB, l, false, 0.0, o.Z, l, st));
  DMD_TRY(dgemm(l, r, r, 1.0, o.Z, l, false, o.Wt, r, false, 0.0, o.Mlift, l, st));
  return DMD_OK;
}

}  // namespace dmd
