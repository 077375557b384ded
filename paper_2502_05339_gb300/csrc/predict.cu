// Exponential-integration prediction and its adjoint (Eq. large_time_step,
// Eq. reverse_simulation, Eq. external_forces; gradients for the inverse
// design use of Sec. 7.2).
//
// Real 2x2-block form: a conjugate pair owning columns (c, c+1) contributes
// Phi_R[:, c] C[c, k] + Phi_R[:, c+1] C[c+1, k] with y = lambda^k zeta,
// zeta = beta_c - i beta_{c+1}, C[c, k] = Re y, C[c+1, k] = -Im y; a real
// eigenvalue's column has C[c, k] = lambda^k beta_c.  lambda^k is evaluated
// in polar form |lambda|^k (cos k theta + i sin k theta), which costs the
// same for every k (negative k included) -- the "arbitrary time step" of the
// paper.
#include "common.cuh"

namespace dmd {

namespace {

// lambda^k for integer k (k = 0 gives exactly 1, also for lambda = 0).
__device__ __forceinline__ void cpow_int(double re, double im, int k, double& pr, double& pi) {
  if (k == 0) {
    pr = 1.0;
    pi = 0.0;
    return;
  }
  const double mag = hypot(re, im);
  if (mag == 0.0) {
    pr = (k > 0) ? 0.0 : INFINITY;
    pi = 0.0;
    return;
  }
  const double th = atan2(im, re);
  const double rk = exp((double)k * log(mag));
  double s, c;
  sincos((double)k * th, &s, &c);
  pr = rk * c;
  pi = rk * s;
}

// C (r x K, ld r) FP64 from the modal buffer and the time indices.
__global__ void k_coefficients(int r, int K, const double* __restrict__ modal, const int32_t* __restrict__ ks,
                               double* __restrict__ C) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * K) return;
  const int c = (int)(t % r);
  const int j = (int)(t / r);
  const double* lre = modal;
  const double* lim = modal + r;
  const double* beta = modal + 2 * r;
  const double li = lim[c];
  if (li < 0.0) return;   // second column of a pair: written by the head
  const int k = ks[j];
  double pr, pi;
  cpow_int(lre[c], li, k, pr, pi);
  if (li > 0.0 && c + 1 < r) {
    const double zr = beta[c], zi = -beta[c + 1];
    const double yr = pr * zr - pi * zi, yi = pr * zi + pi * zr;
    C[(int64_t)j * r + c] = yr;
    C[(int64_t)j * r + c + 1] = -yi;
  } else {
    C[(int64_t)j * r + c] = pr * beta[c];
  }
}

// DMD with control: xi_0 = beta, xi_{t+1} = L xi_t + G_R u_t with L the real
// 2x2-block operator of lambda; writes Xi (r x (steps+1)).  One thread per
// head column; the time loop is sequential, the modes are independent.
// Temporal editing (Eq. edit_temporal): Omega = log(lambda) / dt, cluster by
// |Im Omega| < thr (low) or not (high); lambda' = exp((s_re Re Omega + i s_im
// Im Omega) dt), beta' = w beta; a real eigenvalue keeps its sign.  One
// thread per column; a pair's head writes both columns; sigma and G are
// copied unchanged.
__global__ void k_edit_modes(int r, int q, const double* __restrict__ in, double* __restrict__ out, double thr,
                             double lw, double lre, double lim, double hw, double hre, double him, double dt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r) return;
  out[3 * r + c] = in[3 * r + c];
  for (int j = 0; j < q; ++j) out[4 * r + (int64_t)j * r + c] = in[4 * r + (int64_t)j * r + c];
  const double lr = in[c], li = in[r + c], b = in[2 * r + c];
  if (li < 0.0) return;   // second column of a pair: written by the head
  const double om_re = log(hypot(lr, li)) / dt, om_im = atan2(li, lr) / dt;
  const bool low = fabs(om_im) < thr;
  const double w = low ? lw : hw, sre = low ? lre : hre, sim = low ? lim : him;
  const double mod = exp(sre * om_re * dt);
  if (li > 0.0 && c + 1 < r) {
    double sn, cs;
    sincos(sim * om_im * dt, &sn, &cs);
    out[c] = mod * cs;
    out[r + c] = mod * sn;
    out[c + 1] = mod * cs;
    out[r + c + 1] = -mod * sn;
    out[2 * r + c] = w * b;
    out[2 * r + c + 1] = w * in[2 * r + c + 1];
  } else {
    out[c] = lr >= 0.0 ? mod : -mod;
    out[r + c] = 0.0;
    out[2 * r + c] = w * b;
  }
}

// Upsampling evolution (Sec. 6.3.1) in closed form.  Lambda is diagonal in
// modal coordinates, so the high-order part of R_t = S^L P_t + S^H Lambda
// R_{t-1} is Lambda^t R_0 restricted to the high-order modes, and the
// low-order part is the projection of the input: column t-1 of C (t = 1..T)
// is [P_t on low-order modes; Lambda^t P_0 on the others] in the real form
// (a pair rotates as the prediction coefficients do).  A mode is low-order
// when |Im log(lambda)| / dt < thr.  P is r x (T+1) (column 0 = Phi^+ H_0).
__global__ void k_upsample_coeffs(int r, int T, const double* __restrict__ modal, double thr, double dt,
                                  const double* __restrict__ P, double* __restrict__ C) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)r * T) return;
  const int c = (int)(e % r);
  const int j = (int)(e / r);
  const double lr = modal[c], li = modal[r + c];
  if (li < 0.0) return;   // second column of a pair: written by the head
  const bool pair = li > 0.0 && c + 1 < r;
  const bool low = fabs(atan2(li, lr)) / dt < thr;
  double* out = C + (int64_t)j * r;
  const double* in = P + (int64_t)(j + 1) * r;
  if (low) {
    out[c] = in[c];
    if (pair) out[c + 1] = in[c + 1];
    return;
  }
  double pr, pi;
  cpow_int(lr, li, j + 1, pr, pi);
  if (pair) {
    const double zr = P[c], zi = -P[c + 1];
    out[c] = pr * zr - pi * zi;
    out[c + 1] = -(pr * zi + pi * zr);
  } else {
    out[c] = pr * P[c];
  }
}

__global__ void k_rollout(int r, int q, int steps, const double* __restrict__ modal,
                          const float* __restrict__ u, double* __restrict__ Xi) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r) return;
  const double* lre = modal;
  const double* lim = modal + r;
  const double* beta = modal + 2 * r;
  const double* G = modal + 4 * r;   // r x q
  const double li = lim[c];
  if (li < 0.0) return;
  const bool pair = li > 0.0 && c + 1 < r;
  const double lr = lre[c];
  double a = beta[c], b = pair ? beta[c + 1] : 0.0;
  Xi[c] = a;
  if (pair) Xi[c + 1] = b;
  for (int t = 0; t < steps; ++t) {
    double fa = 0.0, fb = 0.0;
    for (int ch = 0; ch < q; ++ch) {
      const double ut = (double)u[(int64_t)t * q + ch];
      fa = fma(G[(int64_t)ch * r + c], ut, fa);
      if (pair) fb = fma(G[(int64_t)ch * r + c + 1], ut, fb);
    }
    if (pair) {
      const double na = lr * a + li * b + fa;
      const double nb = -li * a + lr * b + fb;
      a = na;
      b = nb;
    } else {
      a = lr * a + fa;
    }
    Xi[(int64_t)(t + 1) * r + c] = a;
    if (pair) Xi[(int64_t)(t + 1) * r + c + 1] = b;
  }
}

// C[:, j] = Xi[:, k_j]
__global__ void k_gather_cols(int r, int K, const double* __restrict__ Xi, const int32_t* __restrict__ ks,
                              int steps, double* __restrict__ C, int32_t* info) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * K) return;
  const int c = (int)(t % r), j = (int)(t / r);
  const int k = ks[j];
  if (k < 0 || k > steps) {
    raise_status(info, DMD_EINVAL, 6000 + j);
    C[t] = 0.0;
    return;
  }
  C[t] = Xi[(int64_t)k * r + c];
}

// Chain rule of the closed-form coefficients (no control): one CTA per
// column; threads stride over the frames; fixed-order block reduction.
__global__ void k_chain_closed(int r, int K, const double* __restrict__ modal, const int32_t* __restrict__ ks,
                               const double* __restrict__ dC, double* __restrict__ dmodal) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const double* lre = modal;
  const double* lim = modal + r;
  const double* beta = modal + 2 * r;
  const double li = lim[c];
  double* dlr = dmodal;
  double* dli = dmodal + r;
  double* db = dmodal + 2 * r;
  if (li < 0.0) return;
  const bool pair = li > 0.0 && c + 1 < r;
  const double lr = lre[c];
  double gzr = 0.0, gzi = 0.0, glr = 0.0, gli = 0.0;
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    const int k = ks[j];
    double pr, pi;
    cpow_int(lr, li, k, pr, pi);
    const double g0 = dC[(int64_t)j * r + c];
    if (pair) {
      const double gr = g0, gi = -dC[(int64_t)j * r + c + 1];   // g = dC_c - i dC_{c+1}
      // conj(lambda^k) g
      gzr += pr * gr + pi * gi;
      gzi += pr * gi - pi * gr;
      if (k != 0) {
        double qr, qi;
        cpow_int(lr, li, k - 1, qr, qi);
        const double zr = beta[c], zi = -beta[c + 1];
        // d = k lambda^{k-1} zeta ; accumulate conj(d) g
        const double dr = k * (qr * zr - qi * zi), di = k * (qr * zi + qi * zr);
        glr += dr * gr + di * gi;
        gli += dr * gi - di * gr;
      }
    } else {
      gzr += pr * g0;
      if (k != 0) {
        double qr, qi;
        cpow_int(lr, 0.0, k - 1, qr, qi);
        glr += k * qr * beta[c] * g0;
      }
    }
  }
  gzr = block_sum(gzr, red);
  gzi = block_sum(gzi, red);
  glr = block_sum(glr, red);
  gli = block_sum(gli, red);
  if (threadIdx.x == 0) {
    if (pair) {
      db[c] = gzr;
      db[c + 1] = -gzi;
      dlr[c] = dlr[c + 1] = glr;
      dli[c] = dli[c + 1] = gli;
    } else {
      db[c] = gzr;
      dlr[c] = glr;
      dli[c] = 0.0;
    }
  }
}

// Reverse recursion of the controlled rollout.  mu_steps = dXi_steps,
// mu_t = L^T mu_{t+1} + dXi_t; dL/du_t = G_R^T mu_{t+1}; dL/dbeta = mu_0;
// dL/dlambda from sum_t mu_{t+1} xi_t^T through the block pattern; dL/dG_R =
// sum_t mu_{t+1} u_t^T.  dXi (r x (steps+1)) holds dL/dxi_t gathered from the
// requested frames.  One thread per head column for mu (modes decouple);
// d_u needs all modes, so it is formed afterwards by k_du from the stored mu.
__global__ void k_rollout_adjoint(int r, int q, int steps, const double* __restrict__ modal,
                                  const float* __restrict__ u, const double* __restrict__ Xi,
                                  const double* __restrict__ dXi, double* __restrict__ Mu,
                                  double* __restrict__ dmodal) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r) return;
  const double* lre = modal;
  const double* lim = modal + r;
  const double li = lim[c];
  if (li < 0.0) return;
  const bool pair = li > 0.0 && c + 1 < r;
  const double lr = lre[c];
  double ma = dXi[(int64_t)steps * r + c];
  double mb = pair ? dXi[(int64_t)steps * r + c + 1] : 0.0;
  Mu[(int64_t)steps * r + c] = ma;
  if (pair) Mu[(int64_t)steps * r + c + 1] = mb;
  double dA = 0.0, dB = 0.0;   // d/dRe lambda, d/dIm lambda
  double* dG = dmodal + 4 * r;
  for (int ch = 0; ch < q; ++ch) {
    dG[(int64_t)ch * r + c] = 0.0;
    if (pair) dG[(int64_t)ch * r + c + 1] = 0.0;
  }
  for (int t = steps - 1; t >= 0; --t) {
    const double xa = Xi[(int64_t)t * r + c];
    const double xb = pair ? Xi[(int64_t)t * r + c + 1] : 0.0;
    // L = [[lr, li], [-li, lr]]: dL/dlr = ma xa + mb xb, dL/dli = ma xb - mb xa
    dA += ma * xa + mb * xb;
    if (pair) dB += ma * xb - mb * xa;
    for (int ch = 0; ch < q; ++ch) {
      const double ut = (double)u[(int64_t)t * q + ch];
      dG[(int64_t)ch * r + c] += ma * ut;
      if (pair) dG[(int64_t)ch * r + c + 1] += mb * ut;
    }
    // mu_t = L^T mu_{t+1} + dXi_t, L^T = [[lr, -li], [li, lr]]
    const double na = (pair ? lr * ma - li * mb : lr * ma) + dXi[(int64_t)t * r + c];
    const double nb = pair ? (li * ma + lr * mb) + dXi[(int64_t)t * r + c + 1] : 0.0;
    ma = na;
    mb = nb;
    Mu[(int64_t)t * r + c] = ma;
    if (pair) Mu[(int64_t)t * r + c + 1] = mb;
  }
  double* dlr = dmodal;
  double* dli = dmodal + r;
  double* db = dmodal + 2 * r;
  db[c] = ma;
  dlr[c] = dA;
  dli[c] = pair ? dB : 0.0;
  if (pair) {
    db[c + 1] = mb;
    dlr[c + 1] = dA;
    dli[c + 1] = dB;
  }
}

// d_u[:, t] = G_R^T mu_{t+1}
__global__ void k_du(int r, int q, int steps, const double* __restrict__ modal, const double* __restrict__ Mu,
                     float* __restrict__ du) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)q * steps) return;
  const int ch = (int)(idx % q), t = (int)(idx / q);
  const double* G = modal + 4 * r;
  double s = 0.0;
  for (int c = 0; c < r; ++c) s = fma(G[(int64_t)ch * r + c], Mu[(int64_t)(t + 1) * r + c], s);
  du[idx] = (float)s;
}

// dXi[:, t] = sum over requested frames j with k_j == t of dC[:, j]; one
// thread per (column, t); frames scanned in order, so the sum is reproducible.
__global__ void k_scatter_frames(int r, int K, int steps, const int32_t* __restrict__ ks,
                                 const double* __restrict__ dC, double* __restrict__ dXi) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)r * (steps + 1)) return;
  const int c = (int)(idx % r), t = (int)(idx / r);
  double s = 0.0;
  for (int j = 0; j < K; ++j)
    if (ks[j] == t) s += dC[(int64_t)j * r + c];
  dXi[idx] = s;
}

// Loss of one chunk: partial[b] = sum over this block's rows of
// sum_j w_j rho(F_ij - tgt_i) with rho(e) = e^2 / 2, or with delta > 0 the
// Huber function (e^2 / 2 for |e| <= delta, delta (|e| - delta / 2) beyond);
// if grad, F <- w_j rho'(F - tgt) in place.
__global__ void k_loss_chunk(int64_t n, int nf, float* __restrict__ F, int64_t ldf, const float* __restrict__ tgt,
                             const double* __restrict__ w, int grad, float delta, double* __restrict__ partial) {
  // Each thread sums its elements of one frame in FP32 (a few dozen terms)
  // and carries the frame sums in FP64: FP64 arithmetic per element would be
  // bound by GB300's FP64 pipe (~64x slower than FP32).
  __shared__ double red[32];
  double loc = 0.0;
  for (int j = 0; j < nf; ++j) {
    const float wj = (float)w[j];
    float* f = F + (int64_t)j * ldf;
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const float d = f[i] - tgt[i], ad = fabsf(d);
      const bool lin = delta > 0.f && ad > delta;
      acc = fmaf(wj, lin ? delta * (ad - 0.5f * delta) : 0.5f * d * d, acc);
      if (grad) f[i] = wj * (lin ? copysignf(delta, d) : d);
    }
    loc += (double)acc;
  }
  const double s = block_sum(loc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(int count, const double* __restrict__ partial, double* __restrict__ out,
                               int accumulate) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < count; ++i) s += partial[i];
  *out = accumulate ? *out + s : s;
}

}  // namespace

dmd_status launch_edit_modes(int r, int q, const double* in, double* out, double thr, const double* low,
                             const double* high, double dt, cudaStream_t st) {
  k_edit_modes<<<(unsigned)ceil_div(r, 128), 128, 0, st>>>(r, q, in, out, thr, low[0], low[1], low[2], high[0],
                                                            high[1], high[2], dt);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_upsample_coeffs(int r, int T, const double* modal, double thr, double dt, const double* P,
                                  double* C, cudaStream_t st) {
  const int64_t total = (int64_t)r * T;
  if (total == 0) return DMD_OK;
  k_upsample_coeffs<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(r, T, modal, thr, dt, P, C);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_coefficients(int r, int K, const double* modal, const int32_t* ks, double* C, cudaStream_t st) {
  const int64_t total = (int64_t)r * K;
  if (total == 0) return DMD_OK;
  k_coefficients<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(r, K, modal, ks, C);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_rollout(int r, int q, int steps, const double* modal, const float* u, double* Xi,
                          cudaStream_t st) {
  k_rollout<<<(unsigned)ceil_div(r, 64), 64, 0, st>>>(r, q, steps, modal, u, Xi);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_gather_cols(int r, int K, const double* Xi, const int32_t* ks, int steps, double* C,
                              int32_t* info, cudaStream_t st) {
  const int64_t total = (int64_t)r * K;
  if (total == 0) return DMD_OK;
  k_gather_cols<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(r, K, Xi, ks, steps, C, info);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_chain_closed(int r, int K, const double* modal, const int32_t* ks, const double* dC,
                               double* dmodal, cudaStream_t st) {
  k_chain_closed<<<(unsigned)r, 128, 0, st>>>(r, K, modal, ks, dC, dmodal);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_rollout_adjoint(int r, int q, int steps, int K, const int32_t* ks, const double* modal,
                                  const float* u, const double* Xi, const double* dC, double* dXi,
                                  double* Mu, double* dmodal, float* du, cudaStream_t st) {
  const int64_t cnt = (int64_t)r * (steps + 1);
  k_scatter_frames<<<(unsigned)ceil_div(cnt, 256), 256, 0, st>>>(r, K, steps, ks, dC, dXi);
  DMD_LAUNCH_CHECK();
  k_rollout_adjoint<<<(unsigned)ceil_div(r, 64), 64, 0, st>>>(r, q, steps, modal, u, Xi, dXi, Mu, dmodal);
  DMD_LAUNCH_CHECK();
  if (du != nullptr && q > 0 && steps > 0) {
    const int64_t tot = (int64_t)q * steps;
    k_du<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(r, q, steps, modal, Mu, du);
    DMD_LAUNCH_CHECK();
  }
  return DMD_OK;
}

int loss_blocks() { return 1024; }

dmd_status launch_loss_chunk(int64_t n, int nf, float* F, int64_t ldf, const float* tgt, const double* w,
                             bool grad, float delta, double* partial, double* loss, bool accumulate, cudaStream_t st) {
  k_loss_chunk<<<loss_blocks(), 256, 0, st>>>(n, nf, F, ldf, tgt, w, grad ? 1 : 0, delta, partial);
  DMD_LAUNCH_CHECK();
  k_sum_partials<<<1, 32, 0, st>>>(loss_blocks(), partial, loss, accumulate ? 1 : 0);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

// out (= or +=) the sum of partial[0 .. count) in index order.
dmd_status launch_sum_partials(int count, const double* partial, double* out, bool accumulate, cudaStream_t st) {
  k_sum_partials<<<1, 32, 0, st>>>(count, partial, out, accumulate ? 1 : 0);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

}  // namespace dmd
