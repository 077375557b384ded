"""DMD with control (Eq. external_forces): GPU fit, controlled rollout and its
adjoint against the FP64 oracle on seeded blob-forced snapshots."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from paper_2502_05339_gb300 import synth
from tests.gpu_util import cols, match, rel

pytestmark = pytest.mark.gpu
BAR = {"fp32": 1e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def scene():
    sc = synth.controlled_scene(24, 2, 5, 80, 3, 2024)
    ref = O.dmdc(sc.X().numpy(), sc.extra["U"], 10)
    return sc, ref


def _fit(dmd, sc, prec):
    Ups = torch.as_tensor(sc.extra["U"].T.astype(np.float32)).contiguous().cuda()   # (m, q)
    model = dmd.dmd_fit(sc.S.cuda(), sc.n, 10, oversample=6, power_iters=1, precision=prec, seed=3, Ups=Ups)
    torch.cuda.synchronize()
    model.check()
    return model


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_dmdc_fit_matches_oracle(dmd, scene, prec):
    sc, ref = scene
    model = _fit(dmd, sc, prec)
    _, err = match(model.lam(), ref["lam"])
    assert err < BAR[prec], err
    # a fresh control sequence: the rolled-out frames of both models agree
    g = np.random.default_rng(5)
    U2 = synth.piecewise_controls(g, 3, 60)
    PhiR_o, beta_o, kinds_o = O.to_real_form(ref["Phi"], ref["lam"], ref["b"])
    L = O.real_block_operator(ref["lam"], kinds_o)
    GR = O.real_form_control(ref["G"], kinds_o)
    Xi = O.rollout_real(L, beta_o, GR, U2, 60)
    Fo = PhiR_o @ Xi
    u = torch.as_tensor(U2.T.astype(np.float32)).contiguous().cuda()   # (steps, q)
    F = cols(dmd.dmd_predict(model, list(range(61)), u=u, precision=prec), sc.n)
    assert rel(F, Fo) < BAR[prec], rel(F, Fo)


def test_dmdc_reproduces_generator(dmd, scene):
    """Noise-free latent generator: the fitted model's response to a new input
    sequence matches the generator's own response."""
    sc, _ = scene
    model = _fit(dmd, sc, "fp32")
    g = np.random.default_rng(9)
    U2 = synth.piecewise_controls(g, 3, 50)
    z = sc.extra["z"][:, 0].copy()
    modes = sc.modes_true.numpy()
    truth = [modes.T @ z]
    for k in range(50):
        z = sc.extra["L"] @ z + sc.extra["PF"] @ U2[:, k]
        truth.append(modes.T @ z)
    truth = np.stack(truth, axis=1)
    u = torch.as_tensor(U2.T.astype(np.float32)).contiguous().cuda()
    F = cols(dmd.dmd_predict(model, list(range(51)), u=u), sc.n)
    assert rel(F, truth) < 1e-5


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_dmdc_adjoint_matches_oracle(dmd, scene, prec):
    """Gradient of ||x_T - x_tgt||^2 w.r.t. u_0..u_{T-1} and beta: the device
    reverse recursion vs the oracle's on the same (device-fitted) model."""
    sc, _ = scene
    model = _fit(dmd, sc, prec)
    T = 40
    g = np.random.default_rng(4)
    U2 = synth.piecewise_controls(g, 3, T)
    u = torch.as_tensor(U2.T.astype(np.float32)).contiguous().cuda()
    x_T = dmd.dmd_predict(model, [T], u=u, precision=prec)
    tgt = torch.zeros_like(x_T)
    tgt[0, : sc.n] = torch.as_tensor(g.standard_normal(sc.n), dtype=torch.float32)
    dOut = (2 * (x_T - tgt)).contiguous()
    dmodal, du = dmd.dmd_predict_backward(model, [T], dOut, u=u, precision=prec)
    # oracle adjoint on the device model's parameters
    r = model.r
    lam = model.lam()
    beta = model.beta()
    kinds = O.pair_kinds(lam)
    GR = model.G()
    PhiR = cols(model.Phi_R, sc.n)
    L = O.real_block_operator(lam, kinds)
    Xi = O.rollout_real(L, beta, GR, U2.astype(np.float64), T)
    dXi = np.zeros_like(Xi)
    dXi[:, T] = PhiR.T @ cols(dOut, sc.n)[:, 0]
    dlr, dli, db, du_o = O.rollout_adjoint(L, GR, Xi, dXi, kinds)
    tol = 1e-5 if prec == "fp32" else 1e-4
    assert rel(du.cpu().numpy().T, du_o) < tol
    dm = dmodal.cpu().numpy()
    assert rel(dm[2 * r:3 * r], db) < tol
    assert rel(dm[:r], dlr) < tol


def test_dmdc_adjoint_central_differences(dmd, scene):
    """The device gradient of L(u, beta) = 0.5 ||x_T - x_tgt||^2 against
    central differences with h = 1e-3 of the same loss evaluated in FP64 for
    the same (device-fitted) model: rollout of the real 2x2-block latent
    recursion, lift by Phi_R.  The loss is quadratic in u and in beta, so the
    differences are exact up to FP64 rounding; the device gradient carries the
    FP32 rounding of its frames: x_T in FP32 differs from the FP64 lift by
    ~1e-7 of x_T, which is ~1e-5 of the residual (the target sits 1e-2 from
    x_T), so every entry of the gradient can be off by ~1e-5 of the
    gradient's largest entry, whatever its own size.  The bar is 1e-3 of the
    entry, with a floor of 1e-4 of the largest entry (10x that level)."""
    sc, _ = scene
    model = _fit(dmd, sc, "fp32")
    T, h = 40, 1e-3
    g = np.random.default_rng(6)
    U2 = synth.piecewise_controls(g, 3, T)                              # (q, T)
    u = torch.as_tensor(U2.T.astype(np.float32)).contiguous().cuda()
    x_T = dmd.dmd_predict(model, [T], u=u, precision="fp32")[0]
    tgt = x_T.clone()
    tgt[: sc.n] += torch.as_tensor(1e-2 * g.standard_normal(sc.n), dtype=torch.float32, device="cuda")
    w = torch.ones(1, dtype=torch.float64, device="cuda")
    _, dmodal, du = dmd.dmd_predict_loss(model, [T], tgt, w, want_grad=True, u=u, precision="fp32")
    du = du.cpu().numpy()                                                # (T, q)
    r = model.r
    dm = dmodal.cpu().numpy()
    lam, beta, GR = model.lam(), model.beta(), model.G()
    kinds = O.pair_kinds(lam)
    L = O.real_block_operator(lam, kinds)
    PhiR = cols(model.Phi_R, sc.n)
    tgt64 = tgt[: sc.n].double().cpu().numpy()
    U64 = U2.astype(np.float32).astype(np.float64)

    def loss(UU, bb):
        Xi = O.rollout_real(L, bb, GR, UU, T)
        res = PhiR @ Xi[:, T] - tgt64
        return 0.5 * float(res @ res)

    for (t, ch) in [(0, 0), (7, 1), (19, 2), (33, 0), (39, 1)]:
        up, um = U64.copy(), U64.copy()
        up[ch, t] += h
        um[ch, t] -= h
        fd = (loss(up, beta) - loss(um, beta)) / (2 * h)
        assert abs(fd - du[t, ch]) <= 1e-3 * max(abs(fd), 1e-1 * np.abs(du).max()), (t, ch, fd, du[t, ch])
    for c in [0, 3, r - 1]:
        bp, bm = beta.copy(), beta.copy()
        bp[c] += h
        bm[c] -= h
        fd = (loss(U64, bp) - loss(U64, bm)) / (2 * h)
        gd = dm[2 * r + c]
        assert abs(fd - gd) <= 1e-3 * max(abs(fd), 1e-1 * np.abs(dm[2 * r:3 * r]).max()), (c, fd, gd)


@pytest.fixture(scope="module")
def scene_cfg2():
    """The DMD-with-control workload's recipe (50 latent pairs, q = 8 blob
    forces, piecewise-constant inputs, the full m = 300) on a 24^3 x 3 grid:
    its weakest latent direction sits at sigma_100 / sigma_1 = 6.4e-6, below
    what the first CholeskyQR pass resolves, so the fit takes the shifted
    fallback."""
    sc = synth.controlled_scene(24, 3, 50, 300, 8, 1002)
    ref = O.dmdc(sc.X().numpy(), sc.extra["U"], 100)
    return sc, ref


# What r = 100 can be graded on.  The recipe's weakest latent direction sits
# at sigma_100 / sigma_1 = 6.4e-6.  The shifted fallback keeps it (the plain
# CholeskyQR2 drops it and the fit ends in DMD_ERANK), but its basis vector is
# formed from the snapshots with coefficients of order sigma_1 / sigma_100, so
# the FP32 partial sums cancel by that factor and the vector carries rounding
# noise near 1e-2 of its norm: measured, the reconstruction of the training
# window is 1e-4 from the FP64 oracle's in both forms, against the oracle's own
# 1e-7 from the data (an orthogonal construction of the basis would be needed
# for FP32 parity of so weak a direction).  The window is graded at 2e-4 in
# both forms.  The rollout of a new input sequence is ill-conditioned in the
# data itself: the oracle's own rollout (200 steps) moves 8.2e-5 when the
# snapshots are perturbed by a relative 1e-7 and 1.3e-2 at 7.6e-6; it is
# graded at 1e-3 (FP32) and 1e-2 (mixed).
WINDOW_BAR = {"fp32": 2e-4, "mixed": 2e-4}
ROLLOUT_BAR = {"fp32": 1e-3, "mixed": 1e-2}


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_dmdc_full_rank_recipe(dmd, scene_cfg2, prec):
    """r = 100 fits (the shifted fallback keeps the weakest latent directions:
    no DMD_ERANK); the reconstruction of the training window with the
    training inputs and the rollout of a new input sequence (200 steps) match
    the FP64 oracle's within WINDOW_BAR and ROLLOUT_BAR (derived above); the
    eigenvalue vector is reported."""
    sc, ref = scene_cfg2
    Ups = torch.as_tensor(sc.extra["U"].T.astype(np.float32)).contiguous().cuda()
    model = dmd.dmd_fit(sc.S.cuda(), sc.n, 100, oversample=10, power_iters=2, precision=prec, seed=1002, Ups=Ups)
    torch.cuda.synchronize()
    model.check()
    lam_g = model.lam()
    perm, worst = match(lam_g, ref["lam"])
    lam_frob = rel(lam_g[perm], ref["lam"])
    PhiR_o, beta_o, kinds_o = O.to_real_form(ref["Phi"], ref["lam"], ref["b"])
    L = O.real_block_operator(ref["lam"], kinds_o)
    GR = O.real_form_control(ref["G"], kinds_o)

    def both(U_in, T, ks):
        Fo = (PhiR_o @ O.rollout_real(L, beta_o, GR, U_in, T))[:, ks]
        u = torch.as_tensor(U_in.T.astype(np.float32)).contiguous().cuda()
        return cols(dmd.dmd_predict(model, ks, u=u, precision=prec), sc.n), Fo

    Fw, Fwo = both(sc.extra["U"], sc.m, list(range(0, sc.m + 1, 10)))
    werr = rel(Fw, Fwo)
    g = np.random.default_rng(12)
    Fr, Fro = both(synth.piecewise_controls(g, 8, 200), 200, list(range(0, 201, 10)))
    rerr = rel(Fr, Fro)
    print(f"[{prec}] r=100: training window {werr:.2e}; new-input rollout {rerr:.2e}; eigenvalue vector "
          f"{lam_frob:.2e} (worst {worst:.2e})")
    assert werr < WINDOW_BAR[prec], werr
    assert rerr < ROLLOUT_BAR[prec], rerr
