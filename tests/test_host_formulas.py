"""Host-side checks of the formulas the device kernels are built on (CPU,
NumPy): the real 2x2 form of the OptDMD Jacobian that the device assembles
from r x r products must give the explicit Jacobian's J^T J, and its J^T rho
must be the gradient of the projected objective of Eq. variable_projection;
the closed-form high-order evolution of the upsampling kernel must equal the
recurrence; the power iterations run on the snapshot Gram must span the
oracle's range finder.  These restate the device formulas independently of
the CUDA code, against the oracle and finite differences."""
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
