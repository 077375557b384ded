"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each checks the oracle against an
independent fact -- brute force on tiny inputs, eigenvalues of a known
generating operator, closed-form identities, invariants, published test
vectors -- chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them (see
test_oracle_mutations.py, which plants such mistakes).
"""
import math

import numpy as np
import pytest

from oracle import dmd_oracle as O
from oracle import philox
from paper_2502_05339_gb300 import synth

GOLDEN = __file__.rsplit("/", 1)[0] + "/golden"


def match_eigs(lam, ref):
    """Greedy minimum-distance matching; returns max |lam_i - ref_j|."""
    ref = list(ref)
    worst = 0.0
    for v in lam:
        j = int(np.argmin([abs(v - t) for t in ref]))
        worst = max(worst, abs(v - ref[j]))
        ref.pop(j)
    return worst


@pytest.fixture(scope="module")
def exact_cfg0():
    sc = synth.config0(noise=0.0, keep_fp64=True)
    return sc, O.exact_dmd(sc.extra["S64"], 20)


# ---------------------------------------------------------------- brute force


def pin_bruteforce(n=12, m=8, r=None, seed=3):
    """Tiny case: exact DMD eigenpairs are eigenpairs of K = X' V_r S_r^-1 U_r^T.

    With r = rank(X) this is the full least-squares operator X' X^+ (Eq.
    reduced_koopman / reduced_koopman_solution); its nonzero spectrum is brute
    forced with a dense n x n eigensolve.
    """
    g = np.random.default_rng(seed)
    S = g.standard_normal((n, m + 1))
    X, Xp = S[:, :m], S[:, 1:]
    r = r or m
    res = O.exact_dmd(S, r)
    if r == m:
        K = Xp @ np.linalg.pinv(X)
    else:
        U, s, Vt = np.linalg.svd(X)
        K = Xp @ Vt[:r].T @ np.diag(1 / s[:r]) @ U[:, :r].T
    ev = np.linalg.eigvals(K)
    ev = ev[np.argsort(-np.abs(ev))][:r]
    assert match_eigs(res["lam"], ev) < 1e-12 * max(1, np.abs(ev).max())
    # exact modes are eigenvectors of the full operator
    Phi, lam = res["Phi"], res["lam"]
    resid = np.linalg.norm(K @ Phi - Phi * lam[None, :]) / np.linalg.norm(Phi)
    assert resid < 1e-11
    # amplitudes: minimum-norm residual, characterised by orthogonality of the
    # residual to range(Phi)
    b = res["b"]
    rvec = Phi @ b - X[:, 0]
    assert np.linalg.norm(Phi.conj().T @ rvec) < 1e-11 * np.linalg.norm(Phi) * np.linalg.norm(X[:, 0])
    # the full operator maps each snapshot to the next exactly when r = rank
    if r == m:
        np.testing.assert_allclose(K @ X, Xp, atol=1e-10)
    return res


def test_bruteforce_full_rank():
    pin_bruteforce(12, 8)


def test_bruteforce_truncated():
    pin_bruteforce(12, 8, r=5)
    pin_bruteforce(10, 6, r=3, seed=11)


def test_reduced_operator_projects_full_operator():
    """A~ = U^T K~ U (Sec. 3.1): the reduced operator is the projection of the
    truncated full operator onto the left singular basis."""
    g = np.random.default_rng(5)
    S = g.standard_normal((30, 11))
    X, Xp = S[:, :10], S[:, 1:]
    r = 6
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    Kt = Xp @ Vt[:r].T @ np.diag(1 / s[:r]) @ U[:, :r].T
    res = O.exact_dmd(S, r)
    Ur = res["U"]
    np.testing.assert_allclose(res["Atilde"], Ur.T @ Kt @ Ur, atol=1e-12)


# ---------------------------------------------------------- known operator


def test_known_operator_eigenvalues(exact_cfg0):
    """Snapshots generated exactly by a linear map with known spectrum return
    that spectrum (cfg0 generator, noise 0) to 1e-10."""
    sc, res = exact_cfg0
    assert match_eigs(res["lam"], sc.lam_true) < 1e-10


def test_known_operator_3d():
    sc = synth.linear_modes_scene(12, 3, 5, 30, 77, keep_fp64=True)
    res = O.exact_dmd(sc.extra["S64"], 10)
    assert match_eigs(res["lam"], sc.lam_true) < 1e-10


def test_known_operator_reconstructs_window(exact_cfg0):
    sc, res = exact_cfg0
    S = sc.extra["S64"]
    F = O.predict(res["Phi"], res["lam"], res["b"], range(S.shape[1]))
    assert np.linalg.norm(F - S) / np.linalg.norm(S) < 1e-11


# ----------------------------------------------------- exponential integration


def test_exponential_integration_equals_operator_power(exact_cfg0):
    """Phi Lambda^k b = X' V S^-1 A~^k W b since W Lambda = A~ W (Eq. large_time_step)."""
    sc, res = exact_cfg0
    S = sc.extra["S64"]
    Xp = S[:, 1:]
    V, s, W, b, At = res["V"], res["s"], res["W"], res["b"], res["Atilde"]
    Wb = W @ b
    Ak = np.eye(At.shape[0], dtype=complex)
    ks = list(range(0, 501))
    F = O.predict(res["Phi"], res["lam"], b, ks)
    lift = Xp @ (V / s[None, :])
    for k in ks:
        ref = (lift @ (Ak @ Wb)).real
        assert np.linalg.norm(F[:, k] - ref) <= 1e-10 * max(np.linalg.norm(ref), 1e-300) + 1e-13
        Ak = At @ Ak


def test_real_form_matches_complex(exact_cfg0):
    sc, res = exact_cfg0
    PhiR, beta, kinds = O.to_real_form(res["Phi"], res["lam"], res["b"])
    ks = [0, 1, 7, 99, 100, 250, 500, -3]
    C = O.coefficients(res["lam"], beta, ks, kinds)
    F = O.predict_real(PhiR, C)
    Fc = O.predict(res["Phi"], res["lam"], res["b"], ks)
    assert np.linalg.norm(F - Fc) / np.linalg.norm(Fc) < 1e-13
    np.testing.assert_allclose(C[:, 0], beta, atol=0)


def test_from_real_form_inverts_real_form():
    """from_real_form turns a real 2x2-block basis back into complex modes.

    Pinned three ways: (a) a basis built by hand, whose complex modes are
    known (a pair's columns (u, v) are the modes u + iv and u - iv, a real
    eigenvalue's column is its mode); (b) the round trip through to_real_form
    of conjugate-closed complex modes; (c) the complex prediction Phi Lambda^k b
    of the recovered modes, with b rebuilt from beta (b = (beta_c - i beta_c+1)/2
    for a pair's first member, its conjugate for the partner), equals the real
    product Phi_R C (Eq. large_time_step)."""
    g = np.random.default_rng(21)
    n = 9
    lam = np.array([0.95 * np.exp(0.4j), 0.95 * np.exp(-0.4j), 0.9 * np.exp(1.1j), 0.9 * np.exp(-1.1j), 0.7, -0.5])
    u, v, p, q, w, z = (g.standard_normal(n) for _ in range(6))
    PhiR = np.stack([u, v, p, q, w, z], axis=1)
    Phi = O.from_real_form(PhiR, lam)
    ref = np.stack([u + 1j * v, u - 1j * v, p + 1j * q, p - 1j * q, w + 0j, z + 0j], axis=1)
    np.testing.assert_array_equal(Phi, ref)
    # (b) round trip of conjugate-closed modes
    a, c = g.standard_normal(n) + 1j * g.standard_normal(n), g.standard_normal(n) + 1j * g.standard_normal(n)
    Phi_c = np.stack([a, a.conj(), c, c.conj(), w + 0j, z + 0j], axis=1)
    b = np.array([0.3 - 0.2j, 0.3 + 0.2j, -1.1 + 0.5j, -1.1 - 0.5j, 0.8, -0.4])
    PhiR2, beta, kinds = O.to_real_form(Phi_c, lam, b)
    np.testing.assert_allclose(O.from_real_form(PhiR2, lam), Phi_c, rtol=0, atol=1e-15)
    # (c) complex prediction with the recovered modes = real-form prediction
    bb = np.zeros(len(lam), dtype=complex)
    for col in range(len(lam)):
        if kinds[col] == 1:
            bb[col] = 0.5 * (beta[col] - 1j * beta[col + 1])
            bb[col + 1] = np.conj(bb[col])
        elif kinds[col] == 0:
            bb[col] = beta[col]
    ks = [0, 1, 5, 40, -3]
    F = O.predict(O.from_real_form(PhiR2, lam), lam, bb, ks)
    Fr = O.predict_real(PhiR2, O.coefficients(lam, beta, ks, kinds))
    np.testing.assert_allclose(F, Fr, rtol=0, atol=1e-12 * np.abs(Fr).max())


def test_int_power_matches_polar():
    z = np.array([0.97 * np.exp(0.3j), 1.01 * np.exp(-2.0j), -0.5 + 0j, 0.8j])
    for k in [0, 1, 2, 3, 17, 500, 1000, -1, -7]:
        np.testing.assert_allclose(O.int_power(z, k), np.abs(z) ** k * np.exp(1j * k * np.angle(z)),
                                   rtol=1e-12)


# ------------------------------------------------------------------ reversal


def test_reversal(exact_cfg0):
    """K~^{-1} = Phi Lambda^{-1} Phi^+ undoes one step (Eq. reverse_simulation),
    and Lambda^{-k} Lambda^k = I on the reduced state."""
    sc, res = exact_cfg0
    Phi, lam, b = res["Phi"], res["lam"], res["b"]
    for k in [1, 5, 60, 200]:
        xk1 = O.predict(Phi, lam, b, [k + 1])[:, 0]
        xk = O.predict(Phi, lam, b, [k])[:, 0]
        z = np.linalg.lstsq(Phi, xk1.astype(complex), rcond=None)[0]
        back = (Phi @ (z / lam)).real
        assert np.linalg.norm(back - xk) < 1e-10 * np.linalg.norm(xk)
        zk = O.int_power(lam, k) * b
        np.testing.assert_allclose(O.int_power(lam, -k) * zk, b, rtol=1e-11, atol=1e-14)
    # backward frames from negative k satisfy the forward step
    xm = O.predict(Phi, lam, b, [-10, -9])
    z = np.linalg.lstsq(Phi, xm[:, 0].astype(complex), rcond=None)[0]
    assert np.linalg.norm((Phi @ (lam * z)).real - xm[:, 1]) < 1e-10 * np.linalg.norm(xm[:, 1])


# --------------------------------------------------------- divergence free


def test_divergence_free_2d(exact_cfg0):
    """C X = 0 implies C Phi = 0 (Sec. 4.5): reconstructions stay divergence-free."""
    sc, res = exact_cfg0
    S = sc.extra["S64"]
    div_in = synth.div2d(__import__("torch").as_tensor(S.T), sc.N).numpy()
    assert np.abs(div_in).max() < 1e-12 * np.abs(S).max()
    F = O.predict(res["Phi"], res["lam"], res["b"], [0, 1, 50, 99, 100, 300, 500])
    import torch
    d = synth.div2d(torch.as_tensor(F.T), sc.N).numpy()
    rel = np.linalg.norm(d, axis=1) / np.linalg.norm(F, axis=0)
    assert rel.max() < 1e-13


def test_divergence_free_3d():
    import torch
    sc = synth.linear_modes_scene(16, 3, 6, 40, 91, keep_fp64=True)
    res = O.exact_dmd(sc.extra["S64"], 12)
    F = O.predict(res["Phi"], res["lam"], res["b"], [0, 3, 39, 40, 120])
    d = synth.div3d(torch.as_tensor(F.T), sc.N).numpy()
    rel = np.linalg.norm(d, axis=1) / np.linalg.norm(F, axis=0)
    assert rel.max() < 1e-13


def test_divergence_detects_non_solenoidal():
    """The divergence check itself is not vacuous."""
    import torch
    g = np.random.default_rng(0)
    x = torch.as_tensor(g.standard_normal(2 * 16 * 16))
    assert float(synth.div2d(x, 16).norm()) > 1.0


# ------------------------------------------------------------------- rSVD


def test_rsvd_exact_when_rank_le_sketch():
    """rSVD with rank(X) <= l reproduces the exact SVD and the exact DMD (Sec. 4.3)."""
    sc = synth.linear_modes_scene(32, 2, 6, 40, 123, keep_fp64=True)   # rank 12
    S = sc.extra["S64"]
    X = S[:, :-1]
    l = 16
    Om = synth.random_sketch(X.shape[1], l, 5)
    for q in (0, 1, 2):
        U, s, V, Q = O.rsvd(X, Om, 12, q)
        Ue, se, Ve = O.svd_truncated(X, 12)
        np.testing.assert_allclose(s, se, rtol=1e-10)
        assert np.linalg.norm(Q.T @ Q - np.eye(l)) < 1e-12
        np.testing.assert_allclose(np.abs(V.T @ Ve), np.eye(12), atol=1e-8)
    ex = O.exact_dmd(S, 12)
    rs = O.rsvd_dmd(S, Om, 12, 1)
    assert match_eigs(rs["lam"], ex["lam"]) < 1e-10
    pe = O.mode_products(*O.to_real_form(ex["Phi"], ex["lam"], ex["b"]))
    pr = O.mode_products(*O.to_real_form(rs["Phi"], rs["lam"], rs["b"]))
    assert np.linalg.norm(pe - pr) / np.linalg.norm(pe) < 1e-9


def test_rsvd_power_iterations_improve_subspace():
    """With a slowly decaying spectrum, power iterations shrink the range error
    (a standard property of the randomized range finder)."""
    g = np.random.default_rng(1)
    U, _ = np.linalg.qr(g.standard_normal((400, 60)))
    V, _ = np.linalg.qr(g.standard_normal((60, 60)))
    s = 1.0 / (1 + np.arange(60)) ** 0.5
    X = U @ np.diag(s) @ V.T
    Om = g.standard_normal((60, 15))
    errs = []
    for q in (0, 1, 3):
        *_, Q = O.rsvd(X, Om, 10, q)
        errs.append(np.linalg.norm(X - Q @ (Q.T @ X), 2))
    assert errs[0] > errs[1] > errs[2] * 0.999
    assert errs[2] < 1.2 * s[15]


# ---------------------------------------------------------------- Philox


def test_philox_published_vectors():
    """Known-answer vectors of Philox4x32-10 (Salmon et al., SC'11; golden file)."""
    rows = [l.split() for l in open(f"{GOLDEN}/philox4x32_10_kat.txt") if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        vals = [int(v, 16) for v in row]
        ctr, key, out = vals[0:4], vals[4:6], vals[6:10]
        assert list(philox.philox4x32_10(ctr, key)) == out


def test_sketch_matrix_is_standard_normal():
    Om = philox.sketch_matrix(200, 40, 1234)
    assert abs(Om.mean()) < 0.03 and abs(Om.std() - 1) < 0.03
    # two Box-Muller outputs of one pair are uncorrelated
    assert abs(np.corrcoef(Om.T.ravel()[0::2], Om.T.ravel()[1::2])[0, 1]) < 0.05
    assert not np.allclose(Om, philox.sketch_matrix(200, 40, 1235))


# --------------------------------------------------------------- adjoint


def _quad_loss_setup(seed=4):
    sc = synth.linear_modes_scene(16, 2, 4, 30, seed, keep_fp64=True)
    res = O.exact_dmd(sc.extra["S64"], 8)
    PhiR, beta, kinds = O.to_real_form(res["Phi"], res["lam"], res["b"])
    g = np.random.default_rng(seed)
    ks = [0, 3, 10, 29, 45]
    tgt = g.standard_normal(PhiR.shape[0])
    w = g.uniform(0, 1, len(ks))
    return res["lam"], beta, kinds, PhiR, ks, tgt, w


def _loss(lam, beta, kinds, PhiR, ks, tgt, w):
    F = O.predict_real(PhiR, O.coefficients(lam, beta, ks, kinds))
    return 0.5 * float(np.sum(w * np.sum((F - tgt[:, None]) ** 2, axis=0)))


def test_adjoint_matches_central_differences():
    """Hand-written adjoint vs central FD (h = 1e-3) on the FP64 forward; for this
    quadratic-in-beta loss FD in beta is exact up to rounding."""
    lam, beta, kinds, PhiR, ks, tgt, w = _quad_loss_setup()
    F = O.predict_real(PhiR, O.coefficients(lam, beta, ks, kinds))
    dF = (F - tgt[:, None]) * w[None, :]
    dC = PhiR.T @ dF
    dlr, dli, db = O.predict_adjoint(lam, beta, ks, dC, kinds)
    h = 1e-3
    for c in range(len(beta)):
        bp, bm = beta.copy(), beta.copy()
        bp[c] += h
        bm[c] -= h
        fd = (_loss(lam, bp, kinds, PhiR, ks, tgt, w) - _loss(lam, bm, kinds, PhiR, ks, tgt, w)) / (2 * h)
        assert abs(fd - db[c]) <= 1e-8 * max(1.0, abs(fd))
    h = 1e-6
    for c in range(len(beta)):
        if kinds[c] == 2:
            continue
        for part, ref in ((1, dlr[c]), (1j, dli[c])):
            if kinds[c] == 0 and part == 1j:
                continue
            lp, lm = lam.copy(), lam.copy()
            lp[c] += h * part
            lm[c] -= h * part
            if kinds[c] == 1:
                lp[c + 1], lm[c + 1] = np.conj(lp[c]), np.conj(lm[c])
            fd = (_loss(lp, beta, kinds, PhiR, ks, tgt, w) - _loss(lm, beta, kinds, PhiR, ks, tgt, w)) / (2 * h)
            assert abs(fd - ref) <= 1e-6 * max(1.0, abs(fd))


def test_frame_loss_closed_forms():
    """Quadratic and Huber per-frame losses on a worked example: frames
    F = [[1, 3], [-2, 0.5]], target (0.5, -1), weights (2, 0.5), delta = 1 give
    residuals [[0.5, 2.5], [-1, 1.5]]; quadratic L = 2 (0.125 + 0.5) +
    0.5 (3.125 + 1.125) = 3.375; Huber L = 2 (0.125 + 0.5) + 0.5 (2 + 1) = 2.75
    (|e| = 1 sits on the boundary, where both pieces give 1/2)."""
    F = np.array([[1.0, 3.0], [-2.0, 0.5]])
    tgt = np.array([0.5, -1.0])
    w = np.array([2.0, 0.5])
    assert O.frame_loss(F, tgt, w) == 3.375
    assert O.frame_loss(F, tgt, w, "huber", 1.0) == 2.75
    np.testing.assert_array_equal(O.frame_loss_grad(F, tgt, w), [[1.0, 1.25], [-2.0, 0.75]])
    np.testing.assert_array_equal(O.frame_loss_grad(F, tgt, w, "huber", 1.0), [[1.0, 0.5], [-2.0, 0.5]])
    # a Huber width above every residual is the quadratic loss; a tiny one is
    # delta * (weighted L1 norm) to first order
    g = np.random.default_rng(11)
    F, tgt, w = g.standard_normal((30, 4)), g.standard_normal(30), g.uniform(0, 1, 4)
    big = 2 * np.abs(F - tgt[:, None]).max()
    assert abs(O.frame_loss(F, tgt, w, "huber", big) - O.frame_loss(F, tgt, w)) <= 1e-13 * O.frame_loss(F, tgt, w)
    np.testing.assert_allclose(O.frame_loss_grad(F, tgt, w, "huber", big), O.frame_loss_grad(F, tgt, w), rtol=0,
                               atol=0)
    d = 1e-9
    l1 = float(np.sum(w[None, :] * np.abs(F - tgt[:, None])))
    assert abs(O.frame_loss(F, tgt, w, "huber", d) / d - l1) <= 1e-6 * l1


def test_huber_adjoint_matches_central_differences_on_a_crop():
    """The Huber loss's gradient through the prediction adjoint (dC = Phi_R^T
    dL/dF, then the FP64 chain rule) against central differences of the FP64
    Huber loss, on a 64-row spatial crop of a fitted model (delta = 0.1 RMS
    of the residual, so both pieces are exercised).  The loss is piecewise
    quadratic in beta, so central differences are exact up to rounding unless
    a residual crosses +-delta within the step."""
    lam, beta, kinds, PhiR, ks, tgt, w = _quad_loss_setup(seed=9)
    rows = np.random.default_rng(2).choice(PhiR.shape[0], 64, replace=False)
    PhiR, tgt = PhiR[rows], tgt[rows]
    F = O.predict_real(PhiR, O.coefficients(lam, beta, ks, kinds))
    delta = 0.1 * float(np.sqrt(np.mean((F - tgt[:, None]) ** 2)))
    E = F - tgt[:, None]
    assert 0.2 < np.mean(np.abs(E) > delta) < 0.98

    def L(lm, bt):
        return O.frame_loss(O.predict_real(PhiR, O.coefficients(lm, bt, ks, kinds)), tgt, w, "huber", delta)

    dC = PhiR.T @ O.frame_loss_grad(F, tgt, w, "huber", delta)
    dlr, dli, db = O.predict_adjoint(lam, beta, ks, dC, kinds)
    h = 1e-7
    for c in range(len(beta)):
        bp, bm = beta.copy(), beta.copy()
        bp[c] += h
        bm[c] -= h
        fd = (L(lam, bp) - L(lam, bm)) / (2 * h)
        assert abs(fd - db[c]) <= 1e-6 * max(1.0, abs(fd)), (c, fd, db[c])
    for c in range(len(beta)):
        if kinds[c] == 2:
            continue
        for part, ref in ((1, dlr[c]), (1j, dli[c])):
            if kinds[c] == 0 and part == 1j:
                continue
            lp, lm = lam.copy(), lam.copy()
            lp[c] += h * part
            lm[c] -= h * part
            if kinds[c] == 1:
                lp[c + 1], lm[c + 1] = np.conj(lp[c]), np.conj(lm[c])
            fd = (L(lp, beta) - L(lm, beta)) / (2 * h)
            assert abs(fd - ref) <= 1e-5 * max(1.0, abs(fd)), (c, part, fd, ref)


# ------------------------------------------------------------------ DMDc


@pytest.fixture(scope="module")
def dmdc_small():
    sc = synth.controlled_scene(16, 2, 4, 60, 2, 31)
    res = O.dmdc(sc.extra["S64"], sc.extra["U"], 8)
    return sc, res


def test_dmdc_recovers_eigenvalues(dmdc_small):
    sc, res = dmdc_small
    assert match_eigs(res["lam"], sc.lam_true) < 1e-10


def test_dmdc_reproduces_controlled_trajectory(dmdc_small):
    """Rolling out z_{k+1} = Lambda z_k + G u_k (Eq. external_forces) from b
    reproduces the training window, and a fresh input sequence reproduces the
    generator's response to it."""
    sc, res = dmdc_small
    S = sc.extra["S64"]
    m = S.shape[1] - 1
    Z = O.dmdc_rollout(res["lam"], res["b"], res["G"], sc.extra["U"], m)
    F = (res["Phi"] @ Z).real
    assert np.linalg.norm(F - S) / np.linalg.norm(S) < 1e-10
    g = np.random.default_rng(9)
    U2 = synth.piecewise_controls(g, 2, 80)
    z = sc.extra["z"][:, 0].copy()
    modes = sc.modes_true.numpy()
    for k in range(80):
        z = sc.extra["L"] @ z + sc.extra["PF"] @ U2[:, k]
    truth = modes.T @ z
    Z2 = O.dmdc_rollout(res["lam"], res["b"], res["G"], U2, 80)
    pred = (res["Phi"] @ Z2[:, -1]).real
    assert np.linalg.norm(pred - truth) / np.linalg.norm(truth) < 1e-9


def test_dmdc_real_form_rollout_and_adjoint(dmdc_small):
    """Real 2x2-block rollout equals the complex one; its reverse recursion
    matches central differences of ||x_T - x_tgt||^2 in u_k and beta."""
    sc, res = dmdc_small
    PhiR, beta, kinds = O.to_real_form(res["Phi"], res["lam"], res["b"])
    L = O.real_block_operator(res["lam"], kinds)
    GR = O.real_form_control(res["G"], kinds)
    U = sc.extra["U"][:, :25]
    T = 25
    Xi = O.rollout_real(L, beta, GR, U, T)
    Zc = O.dmdc_rollout(res["lam"], res["b"], res["G"], U, T)
    np.testing.assert_allclose(PhiR @ Xi, (res["Phi"] @ Zc).real, atol=1e-10)
    g = np.random.default_rng(2)
    tgt = g.standard_normal(PhiR.shape[0])

    def loss(beta_, U_):
        xi = O.rollout_real(L, beta_, GR, U_, T)
        x = PhiR @ xi[:, -1]
        return float(np.sum((x - tgt) ** 2))

    xT = PhiR @ Xi[:, -1]
    dXi = np.zeros_like(Xi)
    dXi[:, -1] = PhiR.T @ (2 * (xT - tgt))
    dlr, dli, db, du = O.rollout_adjoint(L, GR, Xi, dXi, kinds)
    h = 1e-3
    for (i, k) in [(0, 0), (1, 7), (0, 24), (1, 13)]:
        Up, Um = U.copy(), U.copy()
        Up[i, k] += h
        Um[i, k] -= h
        fd = (loss(beta, Up) - loss(beta, Um)) / (2 * h)
        assert abs(fd - du[i, k]) <= 1e-8 * max(1, abs(fd))
    for c in [0, 1, 5]:
        bp, bm = beta.copy(), beta.copy()
        bp[c] += h
        bm[c] -= h
        fd = (loss(bp, U) - loss(bm, U)) / (2 * h)
        assert abs(fd - db[c]) <= 1e-8 * max(1, abs(fd))


# ------------------------------------------------------------- paper table


def test_runtime_table_ratios():
    """Internal consistency of the paper's runtime table (Tab. dmd_runtime):
    754 ms / 8.9 us ~ 84,719x, 754 / 16.15 ~ 47x, 754 / 0.95 ~ 794x."""
    assert round(754e-3 / 8.9e-6) == 84719
    assert round(754 / 16.15) == 47
    assert round(754 / 0.95) == 794


def test_mode_products_match_ground_truth(exact_cfg0):
    """The scale-free per-mode field phi_j b_j equals the generator's
    a_j * phi_true_j (the pair contributes 2 Re(phi b lambda^k))."""
    sc, res = exact_cfg0
    PhiR, beta, kinds = O.to_real_form(res["Phi"], res["lam"], res["b"])
    got = O.mode_products(PhiR, beta, kinds)
    heads = [c for c in range(len(kinds)) if kinds[c] != 2]
    lam_heads = res["lam"][heads]
    modes = sc.modes_true.numpy()
    lam_true = sc.lam_true[0::2]
    for j, lt in enumerate(lam_true):
        c = int(np.argmin(np.abs(lam_heads - lt)))
        truth = sc.amps_true[j] * (modes[2 * j] + 1j * modes[2 * j + 1])
        assert np.linalg.norm(got[:, c] - truth) < 1e-10 * np.linalg.norm(truth)


# ------------------------------------------- exact DMD from inner products


def test_gram_route_known_operator():
    """The inner-product evaluation of exact DMD returns the generating
    spectrum of a noise-free scene, and its mode fields phi_j b_j at sampled
    rows equal the generator's a_j phi_true_j there."""
    sc = synth.linear_modes_scene(12, 3, 5, 30, 78, keep_fp64=True)
    S = sc.extra["S64"]
    rows = np.array([0, 5, 1000, 3001, S.shape[0] - 1])
    res = O.exact_dmd_from_gram(S.T @ S, 10, S[rows, 1:])
    assert match_eigs(res["lam"], sc.lam_true) < 1e-9
    PhiR, beta, kinds = O.to_real_form(res["Phi_rows"], res["lam"], res["b"])
    got = O.mode_products(PhiR, beta, kinds)
    heads = [c for c in range(len(kinds)) if kinds[c] != 2]
    modes = sc.modes_true.numpy()
    for j, lt in enumerate(sc.lam_true[0::2]):
        c = int(np.argmin(np.abs(res["lam"][heads] - lt)))
        truth = sc.amps_true[j] * (modes[2 * j, rows] + 1j * modes[2 * j + 1, rows])
        assert np.linalg.norm(got[:, c] - truth) < 1e-8 * np.linalg.norm(truth)


def test_gram_route_equals_svd_route():
    """On noisy data (full-rank X, truncated at r) the inner-product
    evaluation and the SVD evaluation of the same definition agree."""
    sc = synth.linear_modes_scene(16, 2, 6, 40, 79, noise=1e-3, keep_fp64=True)
    S = sc.extra["S64"]
    r = 12
    ref = O.exact_dmd(S, r)
    rows = np.arange(0, S.shape[0], 7)
    res = O.exact_dmd_from_gram(S.T @ S, r, S[rows, 1:])
    # the inner-product route loses accuracy like eps (sigma_1 / sigma_r)^2
    tol = 100 * np.finfo(float).eps * (ref["s"][0] / ref["s"][-1]) ** 2
    np.testing.assert_allclose(res["s"], ref["s"], rtol=tol)
    assert match_eigs(res["lam"], ref["lam"]) < tol
    k1 = O.pair_kinds(ref["lam"])
    k2 = O.pair_kinds(res["lam"])
    p1 = O.mode_products(*O.to_real_form(ref["Phi"][rows], ref["lam"], ref["b"])[:2], k1)
    p2 = O.mode_products(*O.to_real_form(res["Phi_rows"], res["lam"], res["b"])[:2], k2)
    assert np.linalg.norm(p1 - p2) < tol * np.linalg.norm(p1)


# ----------------------------------------------------------- temporal editing


def test_edit_modes_identity_and_inverse(exact_cfg0):
    """Identity edits return the model; an edit followed by its inverse
    (1/w, 1/s_re, 1/s_im) returns it too."""
    sc, res = exact_cfg0
    PhiR, beta, kinds = O.to_real_form(res["Phi"], res["lam"], res["b"])
    lam = res["lam"]
    l1, b1 = O.edit_modes(lam, beta, 0.3, (1.0, 1.0, 1.0), (1.0, 1.0, 1.0))
    np.testing.assert_allclose(l1, lam, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(b1, beta, rtol=1e-15)
    l2, b2 = O.edit_modes(lam, beta, 0.3, (0.5, 1.5, 0.5), (2.0, 0.5, 1.5))
    l3, b3 = O.edit_modes(l2, b2, 0.3 * 0.5, (2.0, 1 / 1.5, 2.0), (0.5, 2.0, 1 / 1.5))
    np.testing.assert_allclose(l3, lam, rtol=1e-12)
    np.testing.assert_allclose(b3, beta, rtol=1e-14)


def test_edit_modes_closed_forms(exact_cfg0):
    """s_re = 0 removes growth and decay (|lambda'| = 1); s_im = 0 removes the
    oscillation (lambda' real positive); w scales every frame of its cluster
    linearly; the cluster split follows |Im log(lambda)| < threshold."""
    sc, res = exact_cfg0
    PhiR, beta, kinds = O.to_real_form(res["Phi"], res["lam"], res["b"])
    lam = res["lam"]
    l1, _ = O.edit_modes(lam, beta, 1e9, (1.0, 0.0, 1.0), (1.0, 1.0, 1.0))      # everything is "low"
    np.testing.assert_allclose(np.abs(l1), 1.0, rtol=1e-14)
    np.testing.assert_allclose(np.angle(l1), np.angle(lam), rtol=1e-12, atol=1e-14)
    l2, _ = O.edit_modes(lam, beta, 1e9, (1.0, 1.0, 0.0), (1.0, 1.0, 1.0))
    assert np.all(l2.real > 0) and np.all(np.abs(l2.imag) < 1e-15)
    np.testing.assert_allclose(np.abs(l2), np.abs(lam), rtol=1e-14)
    thr = float(np.median(np.abs(np.angle(lam))))
    ks = [0, 3, 17]
    l3, b3 = O.edit_modes(lam, beta, thr, (1.0, 1.0, 1.0), (3.0, 1.0, 1.0))
    high = np.abs(np.angle(lam)) >= thr
    F0 = O.predict_real(PhiR, O.coefficients(lam, beta, ks))
    Fl = O.predict_real(PhiR[:, ~high], O.coefficients(lam[~high], beta[~high], ks))
    F3 = O.predict_real(PhiR, O.coefficients(l3, b3, ks))
    np.testing.assert_allclose(F3, Fl + 3.0 * (F0 - Fl), rtol=1e-10, atol=1e-12 * np.abs(F0).max())


# ------------------------------------------------------------------ OptDMD (Sec. 4.2)

def _exp_data(n=40, T=30, npairs=3, real_eigs=(0.97,), noise=0.0, seed=0):
    """Snapshots x_t = sum_j g_j lambda_j^t (t = 0..T) from known conjugate-closed
    eigenvalues and fields g_j, plus optional Gaussian noise; returns
    (S, lambda, g) with g in the same column order as lambda."""
    g = np.random.default_rng(seed)
    lam_p = np.exp(g.uniform(-0.05, 0.0, npairs) + 1j * g.uniform(0.2, 2.8, npairs))
    fp = g.standard_normal((n, npairs)) + 1j * g.standard_normal((n, npairs))
    lam, fields = [], []
    for j in range(npairs):
        lam += [lam_p[j], np.conj(lam_p[j])]
        fields += [fp[:, j], np.conj(fp[:, j])]
    for a in real_eigs:
        lam.append(complex(a))
        fields.append(g.standard_normal(n) + 0j)
    lam, fields = np.array(lam), np.stack(fields, axis=1)
    t = np.arange(T + 1)
    S = (fields @ (lam[:, None] ** t[None, :])).real
    if noise:
        S = S + noise * np.linalg.norm(S) / math.sqrt(S.size) * g.standard_normal(S.shape)
    return S, lam, fields


def pin_optdmd_noise_free(seed=0):
    """Exponential snapshots are fitted exactly: from eigenvalues perturbed by
    1e-3 the fit returns the generating eigenvalues and the fields
    phi_j b_j = g_j (so that x_t = sum_j phi_j b_j alpha_j^t, t from 0)."""
    S, lam, fields = _exp_data(seed=seed)
    r = len(lam)
    ex = O.exact_dmd(S, r)
    kinds = O.pair_kinds(ex["lam"])
    g = np.random.default_rng(seed + 100)
    lam0 = O.optdmd_alphas(O.optdmd_params(ex["lam"], kinds) + 1e-3 * g.standard_normal(r), kinds)
    res = O.optdmd(S, r, lam0=lam0)
    assert match_eigs(res["lam"], lam) < 1e-9
    prod = res["Phi"] * res["b"][None, :]
    for j in range(r):
        i = int(np.argmin(np.abs(res["lam"] - lam[j])))
        assert np.linalg.norm(prod[:, i] - fields[:, j]) < 1e-8 * np.linalg.norm(fields[:, j]), j
    assert res["f"] < 1e-20 * np.sum(np.abs(res["Y"]) ** 2)


def test_optdmd_noise_free_recovery():
    pin_optdmd_noise_free(0)
    pin_optdmd_noise_free(1)


def test_optdmd_matches_unreduced_least_squares():
    """Variable projection solves the same problem as the unreduced fit over
    (alpha, B) jointly: a general-purpose least-squares solver on
    ||Y - Phi(alpha) B||_F (Vandermonde from numpy.vander, B free complex),
    started from the same eigenvalues, reaches the same alpha and objective."""
    from scipy.optimize import least_squares
    S, lam, _ = _exp_data(n=10, T=25, npairs=2, real_eigs=(), noise=3e-2, seed=5)
    r = 4
    X = S[:, :-1]
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    Y = Vt[:r].T * s[:r][None, :]
    lam0 = O.exact_dmd(S, r)["lam"]
    p_opt, kinds, info = O.optdmd_alpha(Y, lam0, max_evals=400, tol=1e-15)
    assert list(kinds) == [1, 2, 1, 2]
    T = Y.shape[0]

    def alphas(p):
        return np.array([p[0] + 1j * p[1], p[0] - 1j * p[1], p[2] + 1j * p[3], p[2] - 1j * p[3]])

    def resid(x):
        Phi = np.vander(alphas(x[:4]), T, increasing=True).T
        B = (x[4:4 + r * r] + 1j * x[4 + r * r:]).reshape(r, r)
        R = Y - Phi @ B
        return np.concatenate([R.real.ravel(), R.imag.ravel()])

    p0 = np.array([lam0[0].real, lam0[0].imag, lam0[2].real, lam0[2].imag])
    B0 = np.linalg.pinv(np.vander(alphas(p0), T, increasing=True).T) @ Y
    x0 = np.concatenate([p0, B0.real.ravel(), B0.imag.ravel()])
    sol = least_squares(resid, x0, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    f_full = float(sol.fun @ sol.fun)
    assert abs(f_full - info["f"]) <= 1e-8 * info["f"]
    assert np.max(np.abs(sol.x[:4] - p_opt)) < 1e-6
    assert info["f"] < O.varpro_objective(O.optdmd_params(lam0, kinds), kinds, Y)


def test_optdmd_beats_exact_dmd_on_noisy_data():
    """Sec. 4.2's motivation: with noisy snapshots the fit over the whole
    trajectory places the eigenvalues closer to the generating ones than the
    one-step fit of exact DMD (mean over seeds)."""
    e_ex, e_opt = [], []
    for seed in range(6):
        S, lam, _ = _exp_data(n=60, T=80, npairs=3, noise=5e-2, seed=20 + seed)
        r = len(lam)
        e_ex.append(match_eigs(O.exact_dmd(S, r)["lam"], lam))
        e_opt.append(match_eigs(O.optdmd(S, r)["lam"], lam))
    assert np.mean(e_opt) < 0.5 * np.mean(e_ex), (e_opt, e_ex)


def test_optdmd_gram_route_equals_svd_route():
    """The inner-product evaluation of OptDMD (for tall data) returns the same
    eigenvalues, modes and amplitudes as the SVD route on data small enough
    for both."""
    S, lam, _ = _exp_data(n=50, T=40, npairs=3, noise=1e-2, seed=8)
    r = 7
    a = O.optdmd(S, r)
    b = O.optdmd_from_gram(S.T @ S, r, S[:, :-1])
    assert match_eigs(a["lam"], b["lam"]) < 1e-9
    pa = a["Phi"] * a["b"][None, :]
    pb = b["Phi_rows"] * b["b"][None, :]
    for j in range(r):
        i = int(np.argmin(np.abs(b["lam"] - a["lam"][j])))
        assert np.linalg.norm(pb[:, i] - pa[:, j]) < 1e-7 * np.linalg.norm(pa[:, j]), j


# ------------------------------------------------------------ upsampling (Sec. 6.3.1)

def _upsample_setup(seed=3, n=40, npairs=3):
    g = np.random.default_rng(seed)
    lam_p = np.exp(g.uniform(-0.05, 0.0, npairs) + 1j * np.array([0.05, 0.9, 2.0])[:npairs])
    lam, cols = [], []
    for j in range(npairs):
        v = g.standard_normal(n) + 1j * g.standard_normal(n)
        lam += [lam_p[j], np.conj(lam_p[j])]
        cols += [v, np.conj(v)]
    lam.append(0.93 + 0j)
    cols.append(g.standard_normal(n) + 0j)
    return np.array(lam), np.stack(cols, axis=1), g


def test_upsample_reproduces_model_trajectory():
    """Inputs on the model's own trajectory x_t = Phi Lambda^t z: the projection
    of every input equals the evolved state, so any split of the modes returns
    the trajectory (low-order modes from the input, high-order from the
    evolution agree)."""
    lam, Phi, g = _upsample_setup()
    z = g.standard_normal(len(lam)) + 1j * g.standard_normal(len(lam))
    z[1::2][:3] = np.conj(z[0::2][:3])
    traj = np.stack([(Phi @ (lam ** t * z)).real for t in range(9)], axis=1)
    for thr in (0.0, 0.5, 1.5, 10.0):
        H = O.upsample(Phi, lam, traj[:, 0], traj[:, 1:], thr)
        np.testing.assert_allclose(H, traj[:, 1:], atol=1e-10 * np.abs(traj).max())


def test_upsample_all_low_is_orthogonal_projection():
    """Every mode low-order: H_t is the least-squares projection of L_t onto
    the span of the modes (residual orthogonal to every mode)."""
    lam, Phi, g = _upsample_setup()
    L = g.standard_normal((Phi.shape[0], 5))
    H = O.upsample(Phi, lam, L[:, 0], L, threshold=1e9)
    res = L - H
    assert np.abs(Phi.conj().T @ res).max() < 1e-10 * np.abs(L).max()
    # the part of L inside the span is kept exactly
    Lin = np.repeat((Phi @ np.ones(len(lam))).real[:, None], 2, axis=1)
    np.testing.assert_allclose(O.upsample(Phi, lam, Lin[:, 0], Lin, 1e9), Lin, atol=1e-10)


def test_upsample_all_high_is_prediction():
    """No low-order mode (threshold 0): the inputs are ignored and H_t is the
    DMD prediction Phi Lambda^t Phi^+ H_0 (Eq. large_time_step)."""
    lam, Phi, g = _upsample_setup()
    H0 = g.standard_normal(Phi.shape[0])
    L = g.standard_normal((Phi.shape[0], 6))
    H = O.upsample(Phi, lam, H0, L, threshold=0.0)
    z = np.linalg.pinv(Phi) @ H0
    ref = np.stack([(Phi @ (lam ** t * z)).real for t in range(1, 7)], axis=1)
    np.testing.assert_allclose(H, ref, atol=1e-10 * np.abs(ref).max())


def test_upsample_is_linear_and_splits_by_frequency():
    """The map (H_0, L) -> H is linear (Sec. 6.3.1); with a split between the
    modes, the low-order coefficients of H_t follow the input at time t and
    the high-order ones are the evolved initial state."""
    lam, Phi, g = _upsample_setup()
    n = Phi.shape[0]
    a0, a1 = g.standard_normal(n), g.standard_normal(n)
    A, B = g.standard_normal((n, 4)), g.standard_normal((n, 4))
    thr = 0.5                       # low: the pair at 0.05 rad/step and the real mode
    Hab = O.upsample(Phi, lam, 2 * a0 - 3 * a1, 2 * A - 3 * B, thr)
    np.testing.assert_allclose(Hab, 2 * O.upsample(Phi, lam, a0, A, thr) - 3 * O.upsample(Phi, lam, a1, B, thr),
                               atol=1e-10 * np.abs(Hab).max())
    pinv = np.linalg.pinv(Phi)
    low = np.abs(np.angle(lam)) < thr
    z0 = pinv @ a0
    for t in range(4):
        c = pinv @ O.upsample(Phi, lam, a0, A, thr)[:, t]
        np.testing.assert_allclose(c[low], (pinv @ A[:, t])[low], atol=1e-9)
        np.testing.assert_allclose(c[~low], (lam ** (t + 1) * z0)[~low], atol=1e-9)


# ------------------------------------------------------ density advection (Sec. 7.2)

def _uniform_frames(N, dim, vel, K):
    c = N ** dim
    f = np.zeros((dim * c, K))
    for d in range(dim):
        f[d * c:(d + 1) * c, :] = vel[d]
    return f


@pytest.mark.parametrize("dim", [2, 3])
def test_advect_integer_shift_is_roll(dim):
    """A uniform velocity moving one cell per step along every axis shifts the
    density by one cell per step, exactly."""
    N = 8
    g = np.random.default_rng(1)
    rho0 = g.standard_normal((N,) * dim)
    out = O.advect_density(rho0.ravel(), _uniform_frames(N, dim, [1.0] * dim, 3), N, dim, dt=1.0)
    ref = rho0
    for k in range(1, 4):
        ref = np.roll(ref, tuple([1] * dim), axis=tuple(range(dim)))
        np.testing.assert_allclose(out[:, k].reshape((N,) * dim), ref, atol=1e-13)


def test_advect_fractional_shift_is_linear_interpolation():
    """A uniform fractional displacement s = s0 + f (cells) gives
    (1 - f) roll(rho, s0) + f roll(rho, s0 + 1) per axis (2D: the tensor product)."""
    N = 10
    g = np.random.default_rng(2)
    rho0 = g.standard_normal((N, N))
    dt, vel = 0.7, (2.5, -1.2)
    out = O.advect_density(rho0.ravel(), _uniform_frames(N, 2, vel, 1), N, 2, dt=dt)[:, 1].reshape(N, N)
    ref = rho0
    for ax, v in enumerate(vel):
        s = dt * v
        s0 = int(np.floor(s))
        f = s - s0
        ref = (1 - f) * np.roll(ref, s0, axis=ax) + f * np.roll(ref, s0 + 1, axis=ax)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    assert abs(out.sum() - rho0.sum()) < 1e-10            # a uniform shift conserves mass


def test_advect_constant_and_still():
    """A constant density stays constant in any velocity field; zero velocity
    leaves any density unchanged; the centre velocity is the mean of the two
    faces (a field that is +1 and -1 on alternate faces does not move it)."""
    N, dim = 6, 3
    g = np.random.default_rng(3)
    frames = g.standard_normal((dim * N ** dim, 2))
    out = O.advect_density(np.full(N ** dim, 2.5), frames, N, dim, dt=0.8)
    np.testing.assert_allclose(out, 2.5, atol=1e-12)
    rho0 = g.standard_normal(N ** dim)
    np.testing.assert_allclose(O.advect_density(rho0, np.zeros((dim * N ** dim, 2)), N, dim, 0.5)[:, 2], rho0)
    alt = np.zeros((dim * N ** dim, 1))
    ax0 = np.indices((N,) * dim)[0].ravel()
    alt[: N ** dim, 0] = np.where(ax0 % 2 == 0, 1.0, -1.0)
    np.testing.assert_allclose(O.advect_density(rho0, alt, N, dim, 0.9)[:, 1], rho0, atol=1e-13)
