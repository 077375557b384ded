"""Planted mistakes in the oracle (on the CPU) must each fail a pin.

Every mutation below is a plausible slip -- a dropped or swapped term, a wrong
sign or index, a transposed operand -- applied to one oracle function with
monkeypatch; the pins of test_oracle_pins.py are then re-run from scratch and
at least one of them has to fail.
"""
import numpy as np
import pytest

from oracle import dmd_oracle as O
from oracle import philox
from paper_2502_05339_gb300 import synth
import tests.test_oracle_pins as P


def _cfg0_exact():
    sc = synth.config0(noise=0.0, keep_fp64=True)
    return sc, O.exact_dmd(sc.extra["S64"], 20)


def _pins():
    yield lambda: P.pin_bruteforce(12, 8)
    yield lambda: P.pin_bruteforce(12, 8, r=5)
    yield P.test_reduced_operator_projects_full_operator
    fx = _cfg0_exact()
    yield lambda: P.test_known_operator_eigenvalues(fx)
    yield lambda: P.test_known_operator_reconstructs_window(fx)
    yield lambda: P.test_exponential_integration_equals_operator_power(fx)
    yield lambda: P.test_real_form_matches_complex(fx)
    yield lambda: P.test_reversal(fx)
    yield lambda: P.test_mode_products_match_ground_truth(fx)
    yield P.test_int_power_matches_polar
    yield P.test_from_real_form_inverts_real_form
    yield P.test_rsvd_exact_when_rank_le_sketch
    yield P.test_philox_published_vectors
    yield P.test_adjoint_matches_central_differences
    yield P.test_frame_loss_closed_forms
    yield P.test_huber_adjoint_matches_central_differences_on_a_crop
    yield P.test_gram_route_known_operator
    yield P.test_gram_route_equals_svd_route
    yield lambda: P.pin_optdmd_noise_free(0)
    yield P.test_optdmd_matches_unreduced_least_squares
    yield P.test_optdmd_beats_exact_dmd_on_noisy_data
    yield P.test_upsample_reproduces_model_trajectory
    yield P.test_upsample_all_low_is_orthogonal_projection
    yield P.test_upsample_all_high_is_prediction
    yield P.test_upsample_is_linear_and_splits_by_frequency
    yield lambda: P.test_advect_integer_shift_is_roll(2)
    yield lambda: P.test_advect_integer_shift_is_roll(3)
    yield P.test_advect_fractional_shift_is_linear_interpolation
    yield P.test_advect_constant_and_still


def _count_failures():
    fails = 0
    for pin in _pins():
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, ValueError, IndexError):
            fails += 1
    return fails


def _mut_split(S):
    S = np.asarray(S, dtype=np.float64)
    return S[:, :-1], S[:, :-1]                 # X' replaced by X


def _mut_reduced_scale(U, s, V, Xp):
    return (U.T @ Xp @ V) * s[None, :]         # Sigma instead of Sigma^-1


def _mut_reduced_transpose(U, s, V, Xp):
    return ((U.T @ Xp @ V) / s[None, :]).T


def _mut_reduced_rowscale(U, s, V, Xp):
    return (U.T @ Xp @ V) / s[:, None]         # Sigma^-1 on the wrong side


_orig_int_power = O.int_power


def _mut_power(z, k):
    return _orig_int_power(z, k - 1 if k > 0 else k)


_orig_real_form = O.to_real_form


def _mut_real_form(Phi, lam, b):
    PhiR, beta, kinds = _orig_real_form(Phi, lam, b)
    beta = beta.copy()
    beta[kinds == 2] *= -1.0                    # sign of Im(zeta) flipped
    return PhiR, beta, kinds


_orig_coefficients = O.coefficients


def _mut_coefficients(lam, beta, ks, kinds=None):
    C = _orig_coefficients(lam, beta, ks, kinds)
    kk = O.pair_kinds(lam) if kinds is None else kinds
    C[kk == 2] *= -1.0                          # + Im instead of - Im
    return C


_orig_svd = O.svd_truncated


def _mut_svd(X, r):
    U, s, V = _orig_svd(X, r)
    return U[:, ::-1].copy(), s, V             # U columns out of order


def _mut_amplitudes(Phi, x0):
    b, *_ = np.linalg.lstsq(Phi, (1.0001 * x0).astype(complex), rcond=None)
    return b


_orig_adjoint = O.predict_adjoint


def _mut_adjoint(lam, beta, ks, dC, kinds=None):
    a, b, c = _orig_adjoint(lam, np.conj(beta), ks, dC, kinds)
    kk = O.pair_kinds(lam) if kinds is None else kinds
    c = c.copy()
    c[kk == 2] *= -1.0
    return a, b, c


def _mut_from_real_form(PhiR, lam):
    kinds = O.pair_kinds(lam)
    Phi = np.zeros(PhiR.shape, dtype=complex)
    for c in range(PhiR.shape[1]):
        if kinds[c] == 1:
            Phi[:, c] = PhiR[:, c] - 1j * PhiR[:, c + 1]           # Im phi conjugated
            Phi[:, c + 1] = np.conj(Phi[:, c])
        elif kinds[c] == 0:
            Phi[:, c] = PhiR[:, c]
    return Phi


def _mut_from_real_form_partner(PhiR, lam):
    kinds = O.pair_kinds(lam)
    Phi = np.zeros(PhiR.shape, dtype=complex)
    for c in range(PhiR.shape[1]):
        if kinds[c] == 1:
            Phi[:, c] = PhiR[:, c] + 1j * PhiR[:, c + 1]
            Phi[:, c + 1] = Phi[:, c]                               # partner not conjugated
        elif kinds[c] == 0:
            Phi[:, c] = PhiR[:, c]
    return Phi


def _mut_huber_branches(F, tgt, w, kind="quadratic", delta=0.0):
    E = np.asarray(F, dtype=np.float64) - np.asarray(tgt, dtype=np.float64)[:, None]
    if kind == "huber":
        A = np.abs(E)
        rho = np.where(A <= delta, delta * (A - 0.5 * delta), 0.5 * E * E)   # pieces swapped
        return float(np.sum(np.asarray(w)[None, :] * rho))
    return float(np.sum(np.asarray(w)[None, :] * 0.5 * E * E))


_orig_loss_grad = O.frame_loss_grad


def _mut_huber_grad(F, tgt, w, kind="quadratic", delta=0.0):
    if kind == "huber":
        E = np.asarray(F, dtype=np.float64) - np.asarray(tgt, dtype=np.float64)[:, None]
        return np.asarray(w)[None, :] * delta * np.sign(E)                  # clipped everywhere
    return _orig_loss_grad(F, tgt, w, kind, delta)


def _mut_loss_weight(F, tgt, w, kind="quadratic", delta=0.0):
    return _orig_loss_grad(F, tgt, np.sqrt(w), kind, delta)                 # weights not applied linearly


def _mut_philox(ctr, key):
    c = list(ctr)
    c[0], c[2] = c[2], c[0]                     # multipliers on swapped words
    return _orig_philox(c, key)


_orig_philox = philox.philox4x32_10
_orig_mode_products = O.mode_products


def _mut_mode_products(PhiR, beta, kinds):
    return 2.0 * _orig_mode_products(PhiR, beta, kinds)   # dropped the 1/2


_orig_gram_blocks = O.gram_blocks


def _mut_gram_cross(Wg):
    a, b, c, d = _orig_gram_blocks(Wg)
    return a, b.T.copy(), c, d                 # X'^T X instead of X^T X'


def _mut_gram_rhs(Wg):
    a, b, c, d = _orig_gram_blocks(Wg)
    return a, b, c, np.asarray(Wg, dtype=np.float64)[:-1, 0]   # X^T x_0 instead of X'^T x_0


def _mut_vandermonde(alpha, T):
    alpha = np.asarray(alpha, dtype=complex)
    return alpha[None, :] ** np.arange(1, T + 1)[:, None]      # alpha^i instead of alpha^(i-1)


_orig_dparams = O.vandermonde_dparams


def _mut_dparams(p, kinds, T):
    out = _orig_dparams(p, kinds, T)
    for k, D in enumerate(out):
        if kinds[k] == 2:
            out[k] = np.conj(D)                                    # d/d Im with the signs of i swapped
    return out


_orig_optdmd_modes = O.optdmd_modes


def _mut_modes_untransposed(U, Y, p, kinds, info):
    alpha = O.optdmd_alphas(p, kinds)
    B, *_ = np.linalg.lstsq(O.vandermonde(alpha, Y.shape[0]), np.asarray(Y, dtype=complex), rcond=None)
    L = U @ B                                                      # U B instead of U B^T
    b = np.linalg.norm(L, axis=0)
    order = O.canonical_order(alpha)
    return dict(lam=alpha[order], Phi=(L / b[None, :])[:, order], b=b[order].astype(complex), B=B[order],
                Y=Y, U=U, **info)


def _mut_modes_unit_amplitude(U, Y, p, kinds, info):
    out = _orig_optdmd_modes(U, Y, p, kinds, info)
    out["b"] = np.ones_like(out["b"])                              # amplitudes dropped
    return out


def _upsample_variant(swap=False, transpose=False, stale=False):
    def up(Phi, lam, H0, L, threshold, dt=1.0):
        Phi = np.asarray(Phi, dtype=complex)
        lam = np.asarray(lam, dtype=complex)
        low = np.abs(np.log(lam).imag / dt) < threshold

        def proj(x):
            if transpose:
                return Phi.T @ np.asarray(x, dtype=complex)          # Phi^T as printed, Phi not orthogonal
            c, *_ = np.linalg.lstsq(Phi, np.asarray(x, dtype=complex), rcond=None)
            return c

        R = proj(H0)
        out = []
        for t in range(L.shape[1]):
            Rstar = R if stale else lam * R                           # evolution step dropped
            P = proj(L[:, t])
            R = np.where(low, Rstar, P) if swap else np.where(low, P, Rstar)   # S^L and S^H swapped
            out.append((Phi @ R).real)
        return np.stack(out, axis=1)
    return up


def _advect_variant(forward=False, face_only=False, swap_w=False, axis_mix=False):
    def adv(rho0, frames, N, dim, dt):
        shape = (N,) * dim
        c = N ** dim
        rho = np.asarray(rho0, dtype=np.float64).reshape(shape)
        idx = np.meshgrid(*([np.arange(N)] * dim), indexing="ij")
        out = [rho.ravel().copy()]
        for k in range(frames.shape[1]):
            u = np.asarray(frames[:, k], dtype=np.float64)
            pos = []
            for d in range(dim):
                dd = dim - 1 - d if axis_mix else d                   # components read for the wrong axes
                face = u[dd * c:(dd + 1) * c].reshape(shape)
                centre = face if face_only else 0.5 * (face + np.roll(face, -1, axis=d))   # no face average
                pos.append(idx[d] + dt * centre if forward else idx[d] - dt * centre)       # traced forward
            base = [np.floor(p).astype(np.int64) for p in pos]
            frac = [p - b for p, b in zip(pos, base)]
            new = np.zeros(shape)
            for corner in range(1 << dim):
                w = np.ones(shape)
                ix = []
                for d in range(dim):
                    bit = (corner >> d) & 1
                    hi = (1.0 - frac[d]) if swap_w else frac[d]        # interpolation weights swapped
                    w = w * (hi if bit else 1.0 - hi)
                    ix.append((base[d] + bit) % N)
                new += w * rho[tuple(ix)]
            rho = new
            out.append(rho.ravel().copy())
        return np.stack(out, axis=1)
    return adv


MUTATIONS = [
    ("split_snapshots", _mut_split, O),
    ("reduced_operator", _mut_reduced_scale, O),
    ("reduced_operator", _mut_reduced_transpose, O),
    ("reduced_operator", _mut_reduced_rowscale, O),
    ("int_power", _mut_power, O),
    ("to_real_form", _mut_real_form, O),
    ("coefficients", _mut_coefficients, O),
    ("svd_truncated", _mut_svd, O),
    ("amplitudes", _mut_amplitudes, O),
    ("predict_adjoint", _mut_adjoint, O),
    ("philox4x32_10", _mut_philox, philox),
    ("mode_products", _mut_mode_products, O),
    ("frame_loss", _mut_huber_branches, O),
    ("frame_loss_grad", _mut_huber_grad, O),
    ("frame_loss_grad", _mut_loss_weight, O),
    ("from_real_form", _mut_from_real_form, O),
    ("from_real_form", _mut_from_real_form_partner, O),
    ("gram_blocks", _mut_gram_cross, O),
    ("gram_blocks", _mut_gram_rhs, O),
    ("vandermonde", _mut_vandermonde, O),
    ("vandermonde_dparams", _mut_dparams, O),
    ("optdmd_modes", _mut_modes_untransposed, O),
    ("optdmd_modes", _mut_modes_unit_amplitude, O),
    ("upsample", _upsample_variant(swap=True), O),
    ("upsample", _upsample_variant(transpose=True), O),
    ("upsample", _upsample_variant(stale=True), O),
    ("advect_density", _advect_variant(forward=True), O),
    ("advect_density", _advect_variant(face_only=True), O),
    ("advect_density", _advect_variant(swap_w=True), O),
    ("advect_density", _advect_variant(axis_mix=True), O),
]


@pytest.mark.parametrize("name,fn,mod", MUTATIONS, ids=[f"{m[0]}-{i}" for i, m in enumerate(MUTATIONS)])
def test_planted_mistake_is_caught(monkeypatch, name, fn, mod):
    monkeypatch.setattr(mod, name, fn)
    assert _count_failures() >= 1


def test_unmutated_oracle_passes_all_pins():
    assert _count_failures() == 0
