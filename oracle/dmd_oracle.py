"""FP64 CPU oracle for the DMD / DMDc hot path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module; the product path never does.  It shares no code
with the CUDA library: it is a plain, slow, literal restatement of the paper's
equations in NumPy float64, with LAPACK routines (SVD, eig, least squares) as
its only library steps.

Definitions followed (paper sections / equations):

* snapshot matrices X = [x_0 .. x_{m-1}], X' = [x_1 .. x_m]      (Eq. reduced_koopman)
* K = X' V Sigma^{-1} U^T from the rank-r truncated SVD X = U Sigma V^T
                                                                 (Eq. reduced_koopman_solution)
* reduced operator  A~ = U^T X' V Sigma^{-1}                     (Sec. 3.1, text after the solution)
* A~ w_i = lambda_i w_i; exact modes Phi = X' V Sigma^{-1} W     (Sec. 3.1; exact-DMD modes)
* amplitudes z = Phi^+ u  (least squares, not normal equations)  (Eq. projection)
* prediction u(t + k dt) = Phi Lambda^k z(t), any integer k      (Eq. large_time_step)
* reversal  u(t) = Phi Lambda^{-1} z(t + dt)                     (Eq. reverse_simulation)
* randomized SVD: range finder Q with X ~ Q Q^T X, B = Q^T X,
  B = U_B Sigma V^T, X ~ (Q U_B) Sigma V^T                       (Sec. 4.3)
* DMD with control, z(t+dt) = Lambda z(t) + Phi^+ B q(t) dt      (Eq. external_forces)
  with the unknown-B least-squares fit of [A B] (the DMDc the paper cites)
* OptDMD: min over alpha, B of ||conj(V) Sigma - Phi(alpha) B||_F with
  Phi(alpha)_{ij} = alpha_j^(i-1), by variable projection and
  Levenberg-Marquardt; phi_i = U B^T(:, i) / ||U B^T(:, i)||   (Sec. 4.2, Eqs. variable_projection,
                                                                 phi_optdmd)
* temporal editing Omega = log(lambda) / dt, per-cluster scales   (Eq. edit_temporal)
* upsampling R_t = S^L Phi^+ L_t + S^H Lambda R_{t-1}, H_t = Phi R_t  (Sec. 6.3.1)
* density carried by the DMD velocity frames, semi-Lagrangian    (Sec. 7.2)
* streamed per-frame losses (quadratic, Huber) and their frame
  gradients, for the adjoint of the prediction                    (Sec. 7.2)

Readings where the paper is silent or garbled are the ones listed in the
design notes: m+1 snapshot columns, exact (not projected) modes, b = Phi^+ x_0
by least squares, canonical eigenvalue order (|lambda| descending, then Im
descending, conjugate pairs adjacent with Im > 0 first), dt = 1.

Real form.  Prediction treats each conjugate pair as a real 2x2 block: for a
pair (lambda, conj lambda) with mode phi and amplitude b the pair contributes
2 Re(phi lambda^k b) = Re(phi) c0_k + Im(phi) c1_k with
c0_k = Re(lambda^k zeta), c1_k = -Im(lambda^k zeta), zeta = 2 b.  The real
amplitude vector stores beta = (Re zeta, -Im zeta) in the pair's two columns,
so C[:, 0] = beta.  A real eigenvalue keeps one real column with beta = b.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# snapshot matrices, SVD, reduced operator, eigendecomposition
# ----------------------------------------------------------------------------


def split_snapshots(S: np.ndarray):
    """X = S[:, :m], X' = S[:, 1:] for S = [x_0 .. x_m] (Eq. reduced_koopman)."""
    S = np.asarray(S, dtype=np.float64)
    return S[:, :-1], S[:, 1:]


def svd_truncated(X: np.ndarray, r: int):
    """Rank-r thin SVD X ~ U diag(s) V^T (Eq. reduced_koopman_solution).

    Singular values descending; each singular pair's sign is fixed so that the
    largest-magnitude entry of v is positive (signs do not affect lambda, Phi).
    """
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    U, s, V = U[:, :r].copy(), s[:r].copy(), Vt[:r].T.copy()
    piv = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[piv, np.arange(r)])
    sgn[sgn == 0] = 1.0
    return U * sgn, s, V * sgn


def reduced_operator(U: np.ndarray, s: np.ndarray, V: np.ndarray, Xp: np.ndarray) -> np.ndarray:
    """A~ = U^T X' V Sigma^{-1}  (r x r), Sec. 3.1."""
    return (U.T @ Xp @ V) / s[None, :]


def canonical_order(lam: np.ndarray) -> np.ndarray:
    """Permutation: |lambda| descending, then Im descending; each conjugate
    partner placed right after its Im > 0 member; real eigenvalues in place."""
    r = len(lam)
    used = np.zeros(r, dtype=bool)
    heads = [i for i in range(r) if lam[i].imag >= 0.0]
    heads.sort(key=lambda i: (-abs(lam[i]), -lam[i].imag, i))
    order = []
    for i in heads:
        if used[i]:
            continue
        used[i] = True
        order.append(i)
        if lam[i].imag > 0.0:
            cand = [j for j in range(r) if not used[j] and lam[j].imag < 0.0]
            j = min(cand, key=lambda j: abs(lam[j] - np.conj(lam[i])))
            used[j] = True
            order.append(j)
    rest = [i for i in range(r) if not used[i]]   # unmatched Im < 0 (not from real data)
    return np.array(order + rest, dtype=int)


def eig_canonical(A: np.ndarray):
    """Eigenpairs A w = lambda w (Sec. 3.1) in canonical order.

    Each w has unit 2-norm and its largest-magnitude entry real positive.
    """
    lam, W = np.linalg.eig(A)
    order = canonical_order(lam)
    lam, W = lam[order], W[:, order].astype(complex)
    W /= np.linalg.norm(W, axis=0)[None, :]
    piv = np.argmax(np.abs(W), axis=0)
    ph = W[piv, np.arange(W.shape[1])]
    W *= (np.abs(ph) / ph)[None, :]
    return lam, W


def amplitudes(Phi: np.ndarray, x0: np.ndarray) -> np.ndarray:
    """b = Phi^+ x_0 as a least-squares solve (Eq. projection)."""
    b, *_ = np.linalg.lstsq(Phi, x0.astype(complex), rcond=None)
    return b


def exact_dmd(S: np.ndarray, r: int) -> dict:
    """Exact DMD of S = [x_0 .. x_m] at rank r (Sec. 3.1, Eqs. reduced_koopman..projection)."""
    X, Xp = split_snapshots(S)
    U, s, V = svd_truncated(X, r)
    At = reduced_operator(U, s, V, Xp)
    lam, W = eig_canonical(At)
    M = (V / s[None, :]) @ W            # m x r: Phi = X' M
    Phi = Xp @ M
    b = amplitudes(Phi, X[:, 0])
    return dict(U=U, s=s, V=V, Atilde=At, lam=lam, W=W, M=M, Phi=Phi, b=b)


def gram_blocks(Wg: np.ndarray):
    """From Wg = S^T S with S = [x_0 .. x_m] (Eq. reduced_koopman):
    X^T X, X^T X', X'^T X' and X'^T x_0."""
    Wg = np.asarray(Wg, dtype=np.float64)
    return Wg[:-1, :-1], Wg[:-1, 1:], Wg[1:, 1:], Wg[1:, 0]


def exact_dmd_from_gram(Wg: np.ndarray, r: int, Xp_rows: np.ndarray) -> dict:
    """Exact DMD at rank r (same definition as exact_dmd, Sec. 3.1) evaluated
    from inner products, for snapshot matrices too tall to decompose in FP64.

    Inputs: the Gram matrix Wg = S^T S of S = [x_0 .. x_m] ((m+1) x (m+1),
    FP64) and some rows of X' (the modes are returned at those rows only).
    The truncated SVD X = U Sigma V^T is taken from X^T X = V Sigma^2 V^T
    (method of snapshots; U = X V Sigma^{-1} is never formed), so
      A~  = U^T X' V Sigma^{-1} = Sigma^{-1} V^T (X^T X') V Sigma^{-1}
      Phi = X' M with M = V Sigma^{-1} W           (rows of X' only)
      b   solves (M^H X'^T X' M) b = M^H X'^T x_0   (normal equations of Eq. projection).
    Rounding: relative errors grow like eps * (sigma_1 / sigma_r)^2."""
    XtX, XtXp, XptXp, Xptx0 = gram_blocks(Wg)
    ev, V = np.linalg.eigh(XtX)
    idx = np.argsort(ev)[::-1][:r]
    s, V = np.sqrt(ev[idx]), V[:, idx]
    piv = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[piv, np.arange(r)])
    sgn[sgn == 0] = 1.0
    V = V * sgn
    At = (V.T @ XtXp @ V) / s[:, None] / s[None, :]
    lam, W = eig_canonical(At)
    M = (V / s[None, :]) @ W
    G = M.conj().T @ XptXp @ M
    b = np.linalg.solve(G, M.conj().T @ Xptx0)
    Phi_rows = np.asarray(Xp_rows, dtype=np.float64) @ M
    return dict(s=s, V=V, Atilde=At, lam=lam, W=W, M=M, Phi_rows=Phi_rows, b=b)


# ----------------------------------------------------------------------------
# prediction (Eq. large_time_step) and its real 2x2-block form
# ----------------------------------------------------------------------------


def int_power(z: np.ndarray, k: int) -> np.ndarray:
    """z**k for integer k by repeated squaring (k < 0 uses (1/z)**|k|)."""
    z = np.asarray(z, dtype=complex)
    if k < 0:
        z, k = 1.0 / z, -k
    out = np.ones_like(z)
    base = z.copy()
    while k:
        if k & 1:
            out = out * base
        base = base * base
        k >>= 1
    return out


def predict(Phi: np.ndarray, lam: np.ndarray, b: np.ndarray, ks) -> np.ndarray:
    """x_k = Phi Lambda^k b for each k in ks; returns the real part (n x K).

    For real data the eigen-triplets are closed under conjugation, so the
    imaginary part is rounding only.
    """
    D = np.stack([int_power(lam, int(k)) * b for k in ks], axis=1)   # r x K
    return (Phi @ D).real


def pair_kinds(lam: np.ndarray, tol: float = 0.0) -> np.ndarray:
    """Per column: 1 = first of a conjugate pair (Im > 0), 2 = its partner,
    0 = real eigenvalue.  Assumes canonical order."""
    kinds = np.zeros(len(lam), dtype=int)
    i = 0
    while i < len(lam):
        if lam[i].imag > tol and i + 1 < len(lam):
            kinds[i], kinds[i + 1] = 1, 2
            i += 2
        else:
            i += 1
    return kinds


def to_real_form(Phi: np.ndarray, lam: np.ndarray, b: np.ndarray):
    """(Phi_R, beta) of the real 2x2-block form (module docstring)."""
    kinds = pair_kinds(lam)
    n, r = Phi.shape
    PhiR = np.empty((n, r))
    beta = np.empty(r)
    for c in range(r):
        if kinds[c] == 1:
            zeta = 2.0 * b[c]
            PhiR[:, c], PhiR[:, c + 1] = Phi[:, c].real, Phi[:, c].imag
            beta[c], beta[c + 1] = zeta.real, -zeta.imag
        elif kinds[c] == 0:
            PhiR[:, c] = Phi[:, c].real
            beta[c] = b[c].real
    return PhiR, beta, kinds


def coefficients(lam: np.ndarray, beta: np.ndarray, ks, kinds=None) -> np.ndarray:
    """C (r x K): column k is the real-form coefficient vector of Lambda^k b."""
    if kinds is None:
        kinds = pair_kinds(lam)
    r = len(lam)
    C = np.zeros((r, len(ks)))
    for j, k in enumerate(ks):
        pw = int_power(lam, int(k))
        for c in range(r):
            if kinds[c] == 1:
                y = pw[c] * (beta[c] - 1j * beta[c + 1])
                C[c, j], C[c + 1, j] = y.real, -y.imag
            elif kinds[c] == 0:
                C[c, j] = (pw[c] * beta[c]).real
    return C


def edit_modes(lam: np.ndarray, beta: np.ndarray, threshold: float, low, high, dt: float = 1.0):
    """Temporal editing of Eq. edit_temporal.  Omega = log(lambda) / dt; a
    mode belongs to the low-frequency cluster when |Im Omega| < threshold,
    else to the high-frequency one.  Each cluster's edit (w, s_re, s_im)
    gives Omega' = s_re Re Omega + i s_im Im Omega, lambda' = exp(Omega' dt)
    and amplitude w b (beta scales with it in the real form).  Readings: the
    edit is a scale of Re Omega and Im Omega (the paper's factors 0.5 .. 1.5);
    a negative real eigenvalue keeps its sign (only its modulus is edited), so
    the real form stays real.  Conjugate partners get conjugate edits."""
    lam = np.asarray(lam, dtype=complex)
    kinds = pair_kinds(lam)
    out_lam = lam.copy()
    out_beta = np.asarray(beta, dtype=np.float64).copy()
    for c in range(len(lam)):
        if kinds[c] == 2:
            continue
        om = np.log(lam[c]) / dt
        w, sre, sim = low if abs(om.imag) < threshold else high
        if kinds[c] == 0:
            mod = np.exp(sre * om.real * dt)
            out_lam[c] = mod if lam[c].real >= 0 else -mod
            out_beta[c] *= w
            continue
        new = np.exp((sre * om.real + 1j * sim * om.imag) * dt)
        out_lam[c], out_lam[c + 1] = new, np.conj(new)
        out_beta[c] *= w
        out_beta[c + 1] *= w
    return out_lam, out_beta


def upsample(Phi: np.ndarray, lam: np.ndarray, H0: np.ndarray, L: np.ndarray, threshold: float,
             dt: float = 1.0) -> np.ndarray:
    """Upsampling evolution of Sec. 6.3.1 with a DMD basis (Phi, Lambda) of a
    high-resolution simulation, a high-resolution initial state H_0 and
    inputs L_1..L_T (columns of L, n x T, given on the high-resolution grid):
      R_0 = Phi^+ H_0;  for t = 1..T:  R*_t = Lambda R_{t-1},  P_t = Phi^+ L_t,
      R_t = S^L P_t + S^H R*_t,  H_t = Phi R_t.
    S^L keeps the low-order modes (|Im Omega| < threshold, Omega = log(lambda) / dt;
    the paper orders the modes by the size of their imaginary parts and takes
    the low-order ones from the input), S^H the others.  Readings: Phi^+ (least
    squares) where the paper writes Phi^T, since Phi is not orthogonal; the
    low-order set by a frequency threshold as in temporal editing.
    Returns [H_1 .. H_T] (real part, n x T)."""
    Phi = np.asarray(Phi, dtype=complex)
    lam = np.asarray(lam, dtype=complex)
    low = np.abs(np.log(lam).imag / dt) < threshold

    def proj(x):
        c, *_ = np.linalg.lstsq(Phi, np.asarray(x, dtype=complex), rcond=None)
        return c

    R = proj(H0)
    out = []
    for t in range(L.shape[1]):
        Rstar = lam * R
        P = proj(L[:, t])
        R = np.where(low, P, Rstar)
        out.append((Phi @ R).real)
    return np.stack(out, axis=1)


def from_real_form(PhiR: np.ndarray, lam: np.ndarray):
    """Complex modes of a real-form basis (inverse of to_real_form's mode part):
    a pair's columns (Re phi, Im phi) give phi and conj(phi)."""
    kinds = pair_kinds(lam)
    Phi = np.zeros(PhiR.shape, dtype=complex)
    for c in range(PhiR.shape[1]):
        if kinds[c] == 1:
            Phi[:, c] = PhiR[:, c] + 1j * PhiR[:, c + 1]
            Phi[:, c + 1] = np.conj(Phi[:, c])
        elif kinds[c] == 0:
            Phi[:, c] = PhiR[:, c]
    return Phi


def advect_density(rho0: np.ndarray, frames: np.ndarray, N: int, dim: int, dt: float) -> np.ndarray:
    """Density carried by the DMD velocity frames (Sec. 7.2: the velocity from
    the DMD model, the density by classical integration in it).  Semi-
    Lagrangian steps on the periodic MAC grid of the snapshots:
      rho_{k+1}(c) = rho_k(c - dt u_k(c)),
    where u_k(c) is the velocity at the centre of cell c (per axis the mean
    of the two faces around the cell; component d of a frame sits on the low
    d-face of each cell) and rho_k is sampled by multilinear interpolation
    with periodic wrap.  Grid units (cell size 1).  frames: n x K velocity
    frames (n = dim N^dim); returns the densities rho_0..rho_K (N^dim x (K+1))."""
    shape = (N,) * dim
    c = N ** dim
    rho = np.asarray(rho0, dtype=np.float64).reshape(shape)
    idx = np.meshgrid(*([np.arange(N)] * dim), indexing="ij")
    out = [rho.ravel().copy()]
    for k in range(frames.shape[1]):
        u = np.asarray(frames[:, k], dtype=np.float64)
        pos = []
        for d in range(dim):
            face = u[d * c:(d + 1) * c].reshape(shape)
            centre = 0.5 * (face + np.roll(face, -1, axis=d))
            pos.append(idx[d] - dt * centre)
        base = [np.floor(p).astype(np.int64) for p in pos]
        frac = [p - b for p, b in zip(pos, base)]
        new = np.zeros(shape)
        for corner in range(1 << dim):
            w = np.ones(shape)
            ix = []
            for d in range(dim):
                bit = (corner >> d) & 1
                w = w * (frac[d] if bit else 1.0 - frac[d])
                ix.append((base[d] + bit) % N)
            new += w * rho[tuple(ix)]
        rho = new
        out.append(rho.ravel().copy())
    return np.stack(out, axis=1)


def predict_real(PhiR: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Reconstruction as one real product F = Phi_R C."""
    return PhiR @ C


def mode_products(PhiR: np.ndarray, beta: np.ndarray, kinds) -> np.ndarray:
    """Scale-free per-mode fields phi_j b_j (complex, n x #modes with Im >= 0).

    phi b = (Re phi + i Im phi) (beta_c - i beta_{c+1}) / 2 for a pair; phi b for
    a real mode.  Independent of each mode's arbitrary complex scale.
    """
    cols = []
    for c in range(PhiR.shape[1]):
        if kinds[c] == 1:
            phi = PhiR[:, c] + 1j * PhiR[:, c + 1]
            cols.append(phi * (beta[c] - 1j * beta[c + 1]) / 2.0)
        elif kinds[c] == 0:
            cols.append(PhiR[:, c] * beta[c] + 0j)
    return np.stack(cols, axis=1)


# ----------------------------------------------------------------------------
# OptDMD by variable projection (Sec. 4.2, Eqs. variable_projection, phi_optdmd)
# ----------------------------------------------------------------------------


def vandermonde(alpha: np.ndarray, T: int) -> np.ndarray:
    """Phi(alpha) in C^{T x r} with entry (i, j) = alpha_j^(i-1), i = 1..T
    (Eq. variable_projection): row i is time t = i - 1."""
    alpha = np.asarray(alpha, dtype=complex)
    t = np.arange(T)[:, None]
    return alpha[None, :] ** t


def optdmd_params(lam: np.ndarray, kinds) -> np.ndarray:
    """Real parameters p of a conjugate-closed eigenvalue set (canonical
    order): a pair (alpha, conj alpha) in columns c, c+1 is (Re alpha, Im alpha),
    a real eigenvalue is itself.  Reading: for real snapshots the fit keeps
    the eigenvalues closed under conjugation, so B and the modes stay those of
    real data."""
    lam = np.asarray(lam, dtype=complex)
    p = np.zeros(len(lam))
    for c in range(len(lam)):
        if kinds[c] == 1:
            p[c], p[c + 1] = lam[c].real, lam[c].imag
        elif kinds[c] == 0:
            p[c] = lam[c].real
    return p


def optdmd_alphas(p: np.ndarray, kinds) -> np.ndarray:
    """alpha(p): inverse of optdmd_params."""
    alpha = np.zeros(len(p), dtype=complex)
    for c in range(len(p)):
        if kinds[c] == 1:
            alpha[c] = p[c] + 1j * p[c + 1]
            alpha[c + 1] = p[c] - 1j * p[c + 1]
        elif kinds[c] == 0:
            alpha[c] = p[c]
    return alpha


def vandermonde_dparams(p: np.ndarray, kinds, T: int) -> list:
    """d Phi(alpha(p)) / d p_k for every real parameter k (T x r complex each).
    d alpha^t / d alpha = t alpha^(t-1); d alpha / d Re = 1, d alpha / d Im = i
    for the Im > 0 member and -i for its conjugate."""
    alpha = optdmd_alphas(p, kinds)
    t = np.arange(T)[:, None]
    dcol = t * alpha[None, :] ** np.maximum(t - 1, 0)
    out = []
    for k in range(len(p)):
        D = np.zeros((T, len(p)), dtype=complex)
        if kinds[k] == 0:
            D[:, k] = dcol[:, k]
        elif kinds[k] == 1:                      # Re alpha of the pair (k, k+1)
            D[:, k], D[:, k + 1] = dcol[:, k], dcol[:, k + 1]
        else:                                    # Im alpha of the pair (k-1, k)
            D[:, k - 1], D[:, k] = 1j * dcol[:, k - 1], -1j * dcol[:, k]
        out.append(D)
    return out


def varpro_residual(p: np.ndarray, kinds, Y: np.ndarray):
    """For fixed alpha the best B of Eq. variable_projection is the least-squares
    solution B = Phi(alpha)^+ Y; the projected residual is rho = Y - Phi B.
    Returns (rho, Phi, B)."""
    Phi = vandermonde(optdmd_alphas(p, kinds), Y.shape[0])
    B, *_ = np.linalg.lstsq(Phi, Y.astype(complex), rcond=None)
    return Y - Phi @ B, Phi, B


def varpro_objective(p: np.ndarray, kinds, Y: np.ndarray) -> float:
    """||Y - Phi(alpha) B||_F^2 at the best B (Eq. variable_projection, squared)."""
    rho, _, _ = varpro_residual(p, kinds, Y)
    return float(np.sum(np.abs(rho) ** 2))


def varpro_jacobian(p: np.ndarray, kinds, Y: np.ndarray):
    """Residual vector and Jacobian of the projected problem, complex parts
    stacked as real rows.  Column k is -(I - P)(d Phi / d p_k) B with
    P = Phi Phi^+ (Kaufman's form of the variable-projection Jacobian: the
    term it drops is orthogonal to rho, so J^T rho is the exact gradient)."""
    rho, Phi, B = varpro_residual(p, kinds, Y)
    cols = []
    for D in vandermonde_dparams(p, kinds, Y.shape[0]):
        M = D @ B
        C, *_ = np.linalg.lstsq(Phi, M, rcond=None)
        Jk = -(M - Phi @ C)
        cols.append(np.concatenate([Jk.real.ravel(), Jk.imag.ravel()]))
    res = np.concatenate([rho.real.ravel(), rho.imag.ravel()])
    return res, np.stack(cols, axis=1)


def optdmd_alpha(Y: np.ndarray, lam0: np.ndarray, max_evals: int = 40, tol: float = 1e-10,
                 mu0: float = 1e-3):
    """Levenberg-Marquardt on the projected problem, from the eigenvalues lam0
    (canonical order) of a standard DMD solve.  Each step solves
    (J^T J + mu diag(J^T J)) delta = -J^T res at the current point and
    evaluates the objective f = ||res||^2 at p + delta.  The linear model
    predicts the fall pred = -(2 g.delta + delta.J^T J.delta) (g = J^T res).
    A trial that lowers f is taken and mu is scaled by
    max(1/3, 1 - (2 rho - 1)^3) with rho = actual / predicted fall (nu = 2);
    otherwise mu *= nu, nu *= 2 (Nielsen's damping update).  Stops when a taken
    step lowers f by at most tol of it or is below 1e-12 of max |p|, when a
    refused step's predicted fall is at most tol of f, when mu exceeds 1e12,
    or after max_evals objective evaluations (the first one included).
    Returns (p, kinds, info dict)."""
    Y = np.asarray(Y, dtype=np.float64)
    kinds = pair_kinds(np.asarray(lam0, dtype=complex))
    p = optdmd_params(lam0, kinds)
    res, J = varpro_jacobian(p, kinds, Y)
    f = float(res @ res)
    f0, mu, nu, evals, accepted = f, mu0, 2.0, 1, 0
    A, g = J.T @ J, J.T @ res
    while evals < max_evals:
        delta = np.linalg.solve(A + mu * np.diag(np.diag(A)), -g)
        p_new = p + delta
        f_new = varpro_objective(p_new, kinds, Y)
        evals += 1
        pred = -(2.0 * g @ delta + delta @ A @ delta)
        if f_new < f:
            rho = (f - f_new) / pred if pred > 0 else 0.5
            stop = (f - f_new) <= tol * f or np.max(np.abs(delta)) <= 1e-12 * max(1.0, np.max(np.abs(p_new)))
            p, f = p_new, f_new
            mu, nu = mu * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), 2.0
            accepted += 1
            if stop:
                break
            res, J = varpro_jacobian(p, kinds, Y)
            A, g = J.T @ J, J.T @ res
        else:
            stop = pred <= tol * f
            mu, nu = mu * nu, 2.0 * nu
            if stop or mu > 1e12:
                break
    return p, kinds, dict(f0=f0, f=f, evals=evals, accepted=accepted, iters=accepted, mu=mu)


def optdmd(S: np.ndarray, r: int, lam0: np.ndarray | None = None, Omega: np.ndarray | None = None,
           power_iters: int = 2, **lm) -> dict:
    """OptDMD of S = [x_0 .. x_m] at rank r (Sec. 4.2).  X = U Sigma V^T is the
    rank-r SVD of X = [x_0 .. x_{m-1}] (T = m snapshots; the randomized SVD of
    Sec. 4.3 when a test matrix Omega is given); alpha starts from the
    exact-DMD eigenvalues of that SVD (or lam0) and minimises
    ||conj(V) Sigma - Phi(alpha) B||_F.  Modes phi_i = U B^T(:, i) / ||U B^T(:, i)||_2
    (Eq. phi_optdmd) and, as the reading for prediction, amplitudes
    b_i = ||U B^T(:, i)||_2, so that x_t ~ sum_i phi_i b_i alpha_i^t.
    Returned in canonical order."""
    X, _ = split_snapshots(S)
    if Omega is None:
        U, s, V = svd_truncated(X, r)
        if lam0 is None:
            lam0 = exact_dmd(S, r)["lam"]
    else:
        U, s, V, _ = rsvd(X, Omega, r, power_iters)
        if lam0 is None:
            lam0 = rsvd_dmd(S, Omega, r, power_iters)["lam"]
    Y = np.conj(V) * s[None, :]
    p, kinds, info = optdmd_alpha(Y, lam0, **lm)
    return optdmd_modes(U, Y, p, kinds, info)


def optdmd_from_gram(Wg: np.ndarray, r: int, X_rows: np.ndarray, **lm) -> dict:
    """OptDMD (same definition as optdmd, Sec. 4.2) from inner products, for
    snapshot matrices too tall to decompose in FP64: V and Sigma from
    X^T X = V Sigma^2 V^T (Wg = S^T S as in exact_dmd_from_gram), alpha from
    the exact-DMD eigenvalues of the same route, and the modes at some rows
    of X only: U = X V Sigma^{-1} there, U B^T(:, i) at those rows, and
    ||U B^T(:, i)||_2 = ||B(i, :)||_2 because U^T U = I."""
    XtX = gram_blocks(Wg)[0]
    ev, V = np.linalg.eigh(XtX)
    idx = np.argsort(ev)[::-1][:r]
    s, V = np.sqrt(ev[idx]), V[:, idx]
    lam0 = exact_dmd_from_gram(Wg, r, np.zeros((0, XtX.shape[0])))["lam"]
    Y = V * s[None, :]
    p, kinds, info = optdmd_alpha(Y, lam0, **lm)
    alpha = optdmd_alphas(p, kinds)
    B, *_ = np.linalg.lstsq(vandermonde(alpha, Y.shape[0]), Y.astype(complex), rcond=None)
    L = (np.asarray(X_rows, dtype=np.float64) @ (V / s[None, :])) @ B.T
    b = np.linalg.norm(B, axis=1)
    order = canonical_order(alpha)
    return dict(lam=alpha[order], Phi_rows=(L / b[None, :])[:, order], b=b[order].astype(complex), **info)


def optdmd_modes(U: np.ndarray, Y: np.ndarray, p: np.ndarray, kinds, info: dict) -> dict:
    """B = Phi(alpha)^+ Y at the fitted alpha, then Eq. phi_optdmd's modes and
    their norms as amplitudes, in canonical order."""
    alpha = optdmd_alphas(p, kinds)
    B, *_ = np.linalg.lstsq(vandermonde(alpha, Y.shape[0]), np.asarray(Y, dtype=complex), rcond=None)
    L = U @ B.T
    b = np.linalg.norm(L, axis=0)
    Phi = L / b[None, :]
    order = canonical_order(alpha)
    return dict(lam=alpha[order], Phi=Phi[:, order], b=b[order].astype(complex), B=B[order],
                Y=Y, U=U, **info)


# ----------------------------------------------------------------------------
# randomized SVD (Sec. 4.3)
# ----------------------------------------------------------------------------


def rsvd(X: np.ndarray, Omega: np.ndarray, r: int, power_iters: int):
    """Randomized SVD of X with test matrix Omega (m x l), Sec. 4.3.

    Range finder with re-orthonormalisation after every product:
    Q = orth(X Omega); repeat power_iters times: Z = orth(X^T Q), Q = orth(X Z).
    Then B = Q^T X = U_B Sigma V^T and X ~ (Q U_B) Sigma V^T, truncated to r.
    orth() is Householder QR (LAPACK).
    """
    Q, _ = np.linalg.qr(X @ Omega)
    for _ in range(power_iters):
        Z, _ = np.linalg.qr(X.T @ Q)
        Q, _ = np.linalg.qr(X @ Z)
    B = Q.T @ X
    Ub, s, Vt = np.linalg.svd(B, full_matrices=False)
    U, s, V = Q @ Ub[:, :r], s[:r], Vt[:r].T
    piv = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[piv, np.arange(r)])
    sgn[sgn == 0] = 1.0
    return U * sgn, s, V * sgn, Q


def rsvd_dmd(S: np.ndarray, Omega: np.ndarray, r: int, power_iters: int) -> dict:
    """Exact DMD where the SVD of X is the randomized one of Sec. 4.3."""
    X, Xp = split_snapshots(S)
    U, s, V, Q = rsvd(X, Omega, r, power_iters)
    At = reduced_operator(U, s, V, Xp)
    lam, W = eig_canonical(At)
    M = (V / s[None, :]) @ W
    Phi = Xp @ M
    b = amplitudes(Phi, X[:, 0])
    return dict(U=U, s=s, V=V, Q=Q, Atilde=At, lam=lam, W=W, M=M, Phi=Phi, b=b)


# ----------------------------------------------------------------------------
# DMD with control (Eq. external_forces; unknown-B least squares fit)
# ----------------------------------------------------------------------------


def dmdc(S: np.ndarray, Ups: np.ndarray, r: int, p: int | None = None) -> dict:
    """DMDc of S = [x_0..x_m] with inputs Ups = [u_0..u_{m-1}] (q x m).

    [A B] is the least-squares map from Omega = [X; Ups] to X', with Omega's
    SVD truncated to p (input space) and the output space U_hat the rank-r
    left singular vectors of X'.  A~ = U_hat^T X' Vt St^{-1} Ut1^T U_hat,
    A~ W = W Lambda; modes Phi = X' Vt St^{-1} Ut1^T U_hat W; b = Phi^+ x_0;
    the reduced forcing is G = Phi^+ B with B = X' Vt St^{-1} Ut2^T, so that
    z_{k+1} = Lambda z_k + G u_k and x_k = Phi z_k (Eq. external_forces, dt = 1).
    """
    X, Xp = split_snapshots(S)
    n = X.shape[0]
    q = Ups.shape[0]
    if p is None:
        p = r + q
    Om = np.vstack([X, Ups])
    Ut, st, Vt = svd_truncated(Om, p)
    Ut1, Ut2 = Ut[:n], Ut[n:]
    Uh, _, _ = svd_truncated(Xp, r)
    core = Xp @ (Vt / st[None, :])              # n x p
    At = Uh.T @ core @ (Ut1.T @ Uh)            # r x r
    Bt = Uh.T @ core @ Ut2.T                   # r x q
    lam, W = eig_canonical(At)
    Phi = core @ (Ut1.T @ Uh) @ W
    Bfull = core @ Ut2.T                       # n x q
    b = amplitudes(Phi, X[:, 0])
    G, *_ = np.linalg.lstsq(Phi, Bfull.astype(complex), rcond=None)
    return dict(Atilde=At, Btilde=Bt, lam=lam, W=W, Phi=Phi, b=b, G=G, B=Bfull, Uhat=Uh)


def dmdc_rollout(lam: np.ndarray, b: np.ndarray, G: np.ndarray, U: np.ndarray, steps: int) -> np.ndarray:
    """z_0 = b, z_{k+1} = Lambda z_k + G u_k (Eq. external_forces); returns r x (steps+1)."""
    Z = np.empty((len(lam), steps + 1), dtype=complex)
    Z[:, 0] = b
    for k in range(steps):
        Z[:, k + 1] = lam * Z[:, k] + G @ U[:, k]
    return Z


def real_block_operator(lam: np.ndarray, kinds) -> np.ndarray:
    """The real r x r operator L with xi_{k+1} = L xi_k in real-form coordinates.

    For a pair column c: (c0, c1) = (Re y, -Im y) with y -> lambda y, i.e. the
    block [[Re l, Im l], [-Im l, Re l]]; a real eigenvalue is a 1x1 block.
    """
    r = len(lam)
    L = np.zeros((r, r))
    for c in range(r):
        if kinds[c] == 1:
            lr, li = lam[c].real, lam[c].imag
            L[c:c + 2, c:c + 2] = [[lr, li], [-li, lr]]
        elif kinds[c] == 0:
            L[c, c] = lam[c].real
    return L


def real_form_control(G: np.ndarray, kinds) -> np.ndarray:
    """Real-form forcing G_R (r x q): the pair rows are (Re 2g, -Im 2g) like beta."""
    r, q = G.shape
    GR = np.zeros((r, q))
    for c in range(r):
        if kinds[c] == 1:
            GR[c], GR[c + 1] = (2 * G[c]).real, -(2 * G[c]).imag
        elif kinds[c] == 0:
            GR[c] = G[c].real
    return GR


def rollout_real(L: np.ndarray, beta: np.ndarray, GR: np.ndarray, U: np.ndarray, steps: int) -> np.ndarray:
    """xi_0 = beta, xi_{k+1} = L xi_k + G_R u_k; returns r x (steps+1)."""
    Xi = np.empty((len(beta), steps + 1))
    Xi[:, 0] = beta
    for k in range(steps):
        Xi[:, k + 1] = L @ Xi[:, k] + GR @ U[:, k]
    return Xi


# ----------------------------------------------------------------------------
# adjoint of the prediction (gradients for the inverse-design use, Sec. 7.2)
# ----------------------------------------------------------------------------


def predict_adjoint(lam: np.ndarray, beta: np.ndarray, ks, dC: np.ndarray, kinds=None):
    """Gradients of a loss L(C) w.r.t. (Re lambda, Im lambda) and beta.

    dC (r x K) = dL/dC.  For a pair with y_k = lambda^k zeta, zeta = beta_c - i beta_{c+1},
    C[c,k] = Re y_k, C[c+1,k] = -Im y_k, so the real gradient of y_k is
    g_k = dC[c,k] - i dC[c+1,k] and, y being holomorphic in (lambda, zeta),
    dL/dzeta = sum_k conj(lambda^k) g_k, dL/dlambda = sum_k conj(k lambda^{k-1} zeta) g_k
    (each as dRe + i dIm).  Then dbeta_c = Re dL/dzeta, dbeta_{c+1} = -Im dL/dzeta.
    The pair's (Re lambda, Im lambda) gradient is stored in both its columns
    (the conjugate member is tied to the first).  Real modes: C = lambda^k beta.
    """
    if kinds is None:
        kinds = pair_kinds(lam)
    r = len(lam)
    dlam_re, dlam_im, dbeta = np.zeros(r), np.zeros(r), np.zeros(r)
    for c in range(r):
        if kinds[c] == 1:
            zeta = beta[c] - 1j * beta[c + 1]
            gz = 0j
            gl = 0j
            for j, k in enumerate(ks):
                k = int(k)
                g = dC[c, j] - 1j * dC[c + 1, j]
                gz += np.conj(int_power(lam[c:c + 1], k)[0]) * g
                if k != 0:
                    gl += np.conj(k * int_power(lam[c:c + 1], k - 1)[0] * zeta) * g
            dbeta[c], dbeta[c + 1] = gz.real, -gz.imag
            dlam_re[c] = dlam_re[c + 1] = gl.real
            dlam_im[c] = dlam_im[c + 1] = gl.imag
        elif kinds[c] == 0:
            lr = lam[c].real
            for j, k in enumerate(ks):
                k = int(k)
                dbeta[c] += lr ** k * dC[c, j]
                if k != 0:
                    dlam_re[c] += k * lr ** (k - 1) * beta[c] * dC[c, j]
    return dlam_re, dlam_im, dbeta


def rollout_adjoint(L: np.ndarray, GR: np.ndarray, Xi: np.ndarray, dXi: np.ndarray, kinds):
    """Reverse recursion of xi_{k+1} = L xi_k + G_R u_k.

    dXi (r x (T+1)) = dL/dxi_k taken directly by the loss.  mu_T = dXi_T,
    mu_k = L^T mu_{k+1} + dXi_k; dL/du_k = G_R^T mu_{k+1}; dL/dbeta = mu_0;
    dL/dL_block accumulates mu_{k+1} xi_k^T over k and maps to (Re l, Im l)
    through the block pattern [[a, b], [-b, a]].
    """
    r, T1 = Xi.shape
    T = T1 - 1
    mu = dXi[:, T].copy()
    du = np.zeros((GR.shape[1], T))
    dLmat = np.zeros((r, r))
    for k in range(T - 1, -1, -1):
        du[:, k] = GR.T @ mu
        dLmat += np.outer(mu, Xi[:, k])
        mu = L.T @ mu + dXi[:, k]
    dlam_re, dlam_im = np.zeros(r), np.zeros(r)
    for c in range(r):
        if kinds[c] == 1:
            a = dLmat[c, c] + dLmat[c + 1, c + 1]
            bb = dLmat[c, c + 1] - dLmat[c + 1, c]
            dlam_re[c] = dlam_re[c + 1] = a
            dlam_im[c] = dlam_im[c + 1] = bb
        elif kinds[c] == 0:
            dlam_re[c] = dLmat[c, c]
    return dlam_re, dlam_im, mu, du


# ----------------------------------------------------------------------------
# per-frame losses of the streamed objective (Sec. 7.2: gradients of the
# prediction for inverse design; the paper names no loss)
# ----------------------------------------------------------------------------


def frame_loss(F: np.ndarray, tgt: np.ndarray, w: np.ndarray, kind: str = "quadratic", delta: float = 0.0) -> float:
    """L = sum_j w_j sum_i rho(F_ij - tgt_i) for frames F (n x K), one target
    field tgt (n) and frame weights w (K).  rho(e) = e^2 / 2 ("quadratic"), or
    the Huber function of width delta ("huber"): e^2 / 2 for |e| <= delta and
    delta (|e| - delta / 2) beyond (its two pieces meet with equal value and
    slope at |e| = delta)."""
    E = np.asarray(F, dtype=np.float64) - np.asarray(tgt, dtype=np.float64)[:, None]
    if kind == "quadratic":
        rho = 0.5 * E * E
    elif kind == "huber":
        A = np.abs(E)
        rho = np.where(A <= delta, 0.5 * E * E, delta * (A - 0.5 * delta))
    else:
        raise ValueError(kind)
    return float(np.sum(np.asarray(w, dtype=np.float64)[None, :] * rho))


def frame_loss_grad(F: np.ndarray, tgt: np.ndarray, w: np.ndarray, kind: str = "quadratic",
                    delta: float = 0.0) -> np.ndarray:
    """dL/dF (n x K) of frame_loss: w_j rho'(F_ij - tgt_i) with rho'(e) = e, or
    for the Huber function e inside [-delta, delta] and delta sign(e) outside."""
    E = np.asarray(F, dtype=np.float64) - np.asarray(tgt, dtype=np.float64)[:, None]
    if kind == "quadratic":
        d = E
    elif kind == "huber":
        d = np.clip(E, -delta, delta)
    else:
        raise ValueError(kind)
    return np.asarray(w, dtype=np.float64)[None, :] * d
