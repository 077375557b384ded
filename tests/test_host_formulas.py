"""Host-side checks of the formulas the device kernels are built on (CPU,
NumPy): the real 2x2 form of the OptDMD Jacobian that the device assembles
from r x r products must give the explicit Jacobian's J^T J, and its J^T rho
must be the gradient of the projected objective of Eq. variable_projection;
the closed-form high-order evolution of the upsampling kernel must equal the
recurrence; the power iterations run on the snapshot Gram must span the
oracle's range finder; the multishift chain schedule of the Francis kernel
must be a Hessenberg similarity that converges to the eigenvalues.  These
restate the device formulas independently of the CUDA code, against the
oracle, library eigenvalues and finite differences."""
import numpy as np

from oracle import dmd_oracle as O


def _real_basis(p, kinds, T):
    """Phi (Re a^t, Im a^t per pair; a^t per real column) and D (Re, Im of t a^(t-1))."""
    r = len(p)
    t = np.arange(T)
    Phi = np.zeros((T, r))
    D = np.zeros((T, r))
    for c in range(r):
        if kinds[c] == 2:
            continue
        a = complex(p[c], p[c + 1] if kinds[c] == 1 else 0.0)
        z = a ** t
        d = t * a ** np.maximum(t - 1, 0)
        Phi[:, c], D[:, c] = z.real, d.real
        if kinds[c] == 1:
            Phi[:, c + 1], D[:, c + 1] = z.imag, d.imag
    return Phi, D


def _terms(kinds, k):
    if kinds[k] == 0:
        return [(k, k, 1.0)]
    if kinds[k] == 1:
        return [(k, k, 1.0), (k + 1, k + 1, 1.0)]
    return [(k, k - 1, -1.0), (k - 1, k, 1.0)]


def _setup(seed=2, T=40, npairs=3):
    g = np.random.default_rng(seed)
    lam = np.exp(g.uniform(-0.05, 0, npairs) + 1j * g.uniform(0.2, 2.5, npairs))
    lam = np.concatenate([[l, np.conj(l)] for l in lam] + [[0.9 + 0j]])
    kinds = O.pair_kinds(lam)
    p = O.optdmd_params(lam, kinds) + 0.01 * g.standard_normal(len(lam))
    Y = g.standard_normal((T, len(lam)))
    return p, kinds, Y


def test_real_form_jacobian_products_match_explicit_jacobian():
    p, kinds, Y = _setup()
    T, r = Y.shape
    Phi, D = _real_basis(p, kinds, T)
    Pinv = np.linalg.pinv(Phi)
    B = Pinv @ Y
    rho = Y - Phi @ B
    E = D - Phi @ (Pinv @ D)
    # explicit Kaufman Jacobian of the real form, one column per parameter
    J = np.zeros((T * r, r))
    for k in range(r):
        M = np.zeros((T, r))
        for j, i, s in _terms(kinds, k):
            M += s * np.outer(E[:, j], B[i, :])
        J[:, k] = -M.ravel()
    # the device's assembly from Ge = E^T E, Gb = B B^T, Hh = E^T rho B^T
    Ge, Gb, Hh = E.T @ E, B @ B.T, E.T @ rho @ B.T
    JtJ = np.zeros((r, r))
    g = np.zeros(r)
    for k in range(r):
        for (j, i, s) in _terms(kinds, k):
            g[k] -= s * Hh[j, i]
            for l in range(r):
                for (j2, i2, s2) in _terms(kinds, l):
                    JtJ[k, l] += s * s2 * Ge[j, j2] * Gb[i, i2]
    np.testing.assert_allclose(JtJ, J.T @ J, rtol=1e-10, atol=1e-10 * np.abs(JtJ).max())
    np.testing.assert_allclose(g, J.T @ rho.ravel(), rtol=1e-10, atol=1e-12)


def test_real_form_gradient_is_gradient_of_projected_objective():
    """J^T rho (real form) = half the gradient of ||(I - P) Y||^2, which the
    oracle evaluates with the complex Vandermonde (central differences)."""
    p, kinds, Y = _setup(seed=5)
    T, r = Y.shape
    Phi, D = _real_basis(p, kinds, T)
    Pinv = np.linalg.pinv(Phi)
    B = Pinv @ Y
    rho = Y - Phi @ B
    E = D - Phi @ (Pinv @ D)
    Hh = E.T @ rho @ B.T
    g = np.array([-sum(s * Hh[j, i] for j, i, s in _terms(kinds, k)) for k in range(r)])
    h = 1e-6
    fd = np.zeros(r)
    for k in range(r):
        e = np.zeros(r)
        e[k] = h
        fd[k] = (O.varpro_objective(p + e, kinds, Y) - O.varpro_objective(p - e, kinds, Y)) / (2 * h)
    np.testing.assert_allclose(2 * g, fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())


def test_upsample_closed_form_equals_recurrence():
    """High-order modes evolve as Lambda^t R_0 and low-order ones follow the
    input's projection: the real-form coefficients the device forms in one
    pass equal the recurrence of Sec. 6.3.1 run step by step."""
    g = np.random.default_rng(9)
    n, npairs, T = 30, 4, 7
    lam = np.exp(g.uniform(-0.05, 0, npairs) + 1j * np.array([0.05, 0.2, 1.0, 2.5]))
    lam = np.concatenate([[l, np.conj(l)] for l in lam])
    V = g.standard_normal((n, npairs)) + 1j * g.standard_normal((n, npairs))
    Phi = np.concatenate([[V[:, i], np.conj(V[:, i])] for i in range(npairs)]).T
    PhiR = np.zeros((n, 2 * npairs))
    PhiR[:, 0::2], PhiR[:, 1::2] = V.real, V.imag
    H0 = g.standard_normal(n)
    L = g.standard_normal((n, T))
    thr = 0.5
    ref = O.upsample(Phi, lam, H0, L, thr)
    # device form: P = Phi_R^+ [H_0 | L]; column t of C per mode as the kernel writes it
    P = np.linalg.pinv(PhiR) @ np.column_stack([H0, L])
    C = np.zeros((2 * npairs, T))
    for c in range(0, 2 * npairs, 2):
        low = abs(np.angle(lam[c])) < thr
        for j in range(T):
            if low:
                C[c:c + 2, j] = P[c:c + 2, j + 1]
            else:
                y = lam[c] ** (j + 1) * (P[c, 0] - 1j * P[c + 1, 0])
                C[c, j], C[c + 1, j] = y.real, -y.imag
    np.testing.assert_allclose(PhiR @ C, ref, atol=1e-10 * np.abs(ref).max())


def test_gram_space_power_iterations_span_the_range_finder():
    """The fit runs its power iterations on the snapshot Gram W = X^T X: with
    R = chol(Bs^T W Bs) (the first CholeskyQR factor of Y = X Bs), the basis
    Q = X Bs R^-1 has X^T Q = W (Bs R^-1) exactly, so Z = orth(W Bs R^-1) and
    only the last Y = X Z is formed on the tall side.  Its orthonormalised
    range equals that of the oracle's range finder (Sec. 4.3: Q = orth(X
    Omega), then Z = orth(X^T Q), Q = orth(X Z) per power iteration)."""
    g = np.random.default_rng(17)
    n, m, l, q = 3000, 40, 12, 2
    U, _ = np.linalg.qr(g.standard_normal((n, m)))
    V, _ = np.linalg.qr(g.standard_normal((m, m)))
    X = (U * np.logspace(0, -3, m)) @ V.T
    Omega = g.standard_normal((m, l))
    *_, Q_ref = O.rsvd(X, Omega, l, q)
    W = X.T @ X
    Bs = Omega
    for _ in range(q):
        R = np.linalg.cholesky(Bs.T @ W @ Bs).T            # upper: Bs^T W Bs = R^T R
        M = np.linalg.solve(R.T, Bs.T).T                   # Bs R^-1
        Zp = W @ M
        np.testing.assert_allclose(Zp, X.T @ (X @ M), atol=1e-12 * np.abs(Zp).max())
        Bs, _ = np.linalg.qr(Zp)                            # the small-space orthonormalisation
    R = np.linalg.cholesky(Bs.T @ W @ Bs).T
    Q = X @ np.linalg.solve(R.T, Bs.T).T                   # the one tall sketch, first pass
    np.testing.assert_allclose(Q.T @ Q, np.eye(l), atol=1e-9)
    np.testing.assert_allclose(Q @ Q.T, Q_ref @ Q_ref.T, atol=1e-9)


def _refl3(x, y, z):
    """P = I - tau v v^T, v = (1, v1, v2), P (x, y, z) = (beta, 0, 0)."""
    nrm = np.sqrt(x * x + y * y + z * z)
    if nrm == 0.0 or (y == 0.0 and z == 0.0):
        return None
    beta = nrm if x <= 0 else -nrm
    return (beta - x) / beta, y / (x - beta), z / (x - beta)


def _apply_rows(H, k, nr, c0, c1, P, zc):
    tau, v1, v2 = P
    v = np.array([1.0, v1, v2])[:nr]
    blk = H[k:k + nr, c0:c1 + 1]
    blk -= tau * np.outer(v, v @ blk)
    if zc >= 0:
        H[k + 1:k + nr, zc] = 0.0


def _apply_cols(H, k, nr, r0, r1, P):
    tau, v1, v2 = P
    v = np.array([1.0, v1, v2])[:nr]
    blk = H[r0:r1 + 1, k:k + nr]
    blk -= tau * np.outer(blk @ v, v)


def _chain_sweep(H, lo, hi, shifts):
    """One chain of small bulges over window [lo, hi] in the kernel's order:
    bulge j (shift sum and product shifts[j]) enters at step 3 j; each step
    forms every bulge's reflector from the current matrix, applies all of
    them from the left, then all from the right."""
    s = len(shifts)
    for t in range((hi - 1 - lo) + 3 * (s - 1) + 1):
        steps = []
        for j, (ss, tt) in enumerate(shifts):
            k = lo + t - 3 * j
            if k < lo or k > hi - 1:
                continue
            nr = 3 if k <= hi - 2 else 2
            if k == lo:
                h = H
                x = h[lo, lo] ** 2 + h[lo, lo + 1] * h[lo + 1, lo] - ss * h[lo, lo] + tt
                y = h[lo + 1, lo] * (h[lo, lo] + h[lo + 1, lo + 1] - ss)
                z = h[lo + 1, lo] * h[lo + 2, lo + 1]
            else:
                x, y = H[k, k - 1], H[k + 1, k - 1]
                z = H[k + 2, k - 1] if nr == 3 else 0.0
            P = _refl3(x, y, z if nr == 3 else 0.0)
            if P is not None:
                steps.append((k, nr, P))
        for k, nr, P in steps:
            _apply_rows(H, k, nr, max(lo, k - 1), hi, P, k - 1 if k > lo else -1)
        for k, nr, P in steps:
            _apply_cols(H, k, nr, lo, min(k + 3, hi), P)


def test_multishift_chain_is_a_hessenberg_similarity():
    """The schedule of the FP32 Francis kernel (bulges three rows apart, all
    reflectors of a step applied from the left, then all from the right):
    one chain sweep over an unreduced Hessenberg matrix keeps it upper
    Hessenberg and is an orthogonal similarity (eigenvalues and Frobenius
    norm kept), and repeated sweeps with the trailing block's eigenvalues as
    shifts deflate the matrix to its eigenvalues."""
    g = np.random.default_rng(23)
    n = 48
    A = g.standard_normal((n, n))
    H0 = np.triu(A, -1)
    H = H0.copy()
    _chain_sweep(H, 0, n - 1, [(0.3, 0.5), (-0.2, 0.8), (1.1, 0.4), (0.0, 1.0)])
    assert np.abs(np.tril(H, -2)).max() < 1e-12 * np.abs(H0).max()
    np.testing.assert_allclose(np.linalg.norm(H), np.linalg.norm(H0), rtol=1e-12)
    ev = np.sort_complex(np.linalg.eigvals(H))
    np.testing.assert_allclose(ev, np.sort_complex(np.linalg.eigvals(H0)), atol=1e-9)
    # the iteration: 8 shifts from the trailing 8 x 8 block, deflation at 1e-12
    H = H0.copy()
    found = []
    hi = n - 1
    for _ in range(400):
        if hi < 0:
            break
        lo = hi
        while lo > 0 and abs(H[lo, lo - 1]) > 1e-12 * (abs(H[lo - 1, lo - 1]) + abs(H[lo, lo])):
            lo -= 1
        if lo > 0:
            H[lo, lo - 1] = 0.0
        if lo == hi:
            found.append(H[hi, hi] + 0j)
            hi -= 1
            continue
        if lo == hi - 1:
            found += list(np.linalg.eigvals(H[hi - 1:hi + 1, hi - 1:hi + 1]))
            hi -= 2
            continue
        if hi - lo + 1 >= 12:
            mu = np.linalg.eigvals(H[hi - 7:hi + 1, hi - 7:hi + 1])
            mu = mu[np.argsort(mu.imag)]                     # conjugates pair up (-im, +im)...
            shifts = []
            cplx = sorted([z for z in mu if z.imag > 0], key=lambda z: z.real)
            real = sorted([z.real for z in mu if z.imag == 0])
            shifts += [(2 * z.real, abs(z) ** 2) for z in cplx]
            shifts += [(real[i] + real[i + 1], real[i] * real[i + 1]) for i in range(0, len(real) - 1, 2)]
            _chain_sweep(H, lo, hi, shifts)
        else:
            a, b, c, d = H[hi - 1, hi - 1], H[hi - 1, hi], H[hi, hi - 1], H[hi, hi]
            _chain_sweep(H, lo, hi, [(a + d, a * d - b * c)])
    assert hi < 0
    np.testing.assert_allclose(np.sort_complex(np.array(found)), np.sort_complex(np.linalg.eigvals(H0)),
                               atol=1e-8)
