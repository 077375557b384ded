"""End-to-end parity of the fit (rSVD + FP64 small solvers) and prediction
against the exact-SVD FP64 oracle, on seeded synthetic snapshots."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from paper_2502_05339_gb300 import synth
from tests.gpu_util import cols, match, mode_product_error, oracle_model, rel

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "mixed"]
BAR = {"fp32": 1e-5, "mixed": 1e-4}   # relative Frobenius error bars
# ||div x_k|| / ||x_k|| of a reconstruction of divergence-free data: the frames
# carry the GEMM rounding of their precision (about sqrt(depth) * u), and the
# divergence is a 4-point difference of it; 10x that level is the bar.
DIV_BAR = {"fp32": 1e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def cfg0():
    sc = synth.config0()
    ref, PhiR, beta, kinds = oracle_model(sc.X().numpy(), 20)
    return sc, ref, PhiR, beta


def _fit(dmd, sc, r, prec, oversample=10, power_iters=2, seed=5):
    model = dmd.dmd_fit(sc.S.cuda(), sc.n, r, oversample=oversample, power_iters=power_iters,
                        precision=prec, seed=seed)
    torch.cuda.synchronize()
    model.check()
    return model


@pytest.mark.parametrize("prec", PRECS)
def test_cfg0_fit_and_predict(dmd, cfg0, prec):
    """Config 0 (2D 64x64, m = 100, r = 20, k = 0..500): eigenvalues, per-mode
    fields phi_j b_j and all 501 frames within the bar."""
    sc, ref, PhiR_o, beta_o = cfg0
    model = _fit(dmd, sc, 20, prec)
    lam_g = model.lam()
    _, lam_err = match(lam_g, ref["lam"])
    assert lam_err < BAR[prec], lam_err
    PhiR_g = cols(model.Phi_R, sc.n)
    mp_frob, mp = mode_product_error(PhiR_g, model.beta(), lam_g, PhiR_o, beta_o, ref["lam"])
    assert mp_frob < BAR[prec], (mp_frob, mp)
    ks = list(range(0, 501))
    F = dmd.dmd_predict(model, ks, precision=prec)
    Fo = O.predict_real(PhiR_o, O.coefficients(ref["lam"], beta_o, ks))
    Fg = cols(F, sc.n)
    inwin = rel(Fg[:, :100], Fo[:, :100])
    allf = rel(Fg, Fo)
    assert inwin < BAR[prec], inwin
    assert allf < BAR[prec], allf
    np.testing.assert_allclose(model.sigma(), ref["s"], rtol=BAR[prec])


@pytest.mark.parametrize("prec", PRECS)
def test_known_operator_gpu(dmd, prec):
    """Noise-free snapshots of a known linear map return its eigenvalues (to the
    FP32 rounding of the stored snapshots)."""
    sc = synth.config0(noise=0.0)
    model = _fit(dmd, sc, 20, prec)
    _, err = match(model.lam(), sc.lam_true)
    assert err < (1e-6 if prec == "fp32" else 1e-5), err


@pytest.mark.parametrize("prec", PRECS)
def test_rsvd_equals_exact_when_rank_fits_sketch(dmd, prec):
    """rank(X) = 12 <= l = 16: the randomized fit equals the exact one."""
    sc = synth.linear_modes_scene(32, 2, 6, 40, 123)
    ref, PhiR_o, beta_o, _ = oracle_model(sc.X().numpy(), 12)
    model = _fit(dmd, sc, 12, prec, oversample=4, power_iters=0)
    _, err = match(model.lam(), ref["lam"])
    assert err < BAR[prec]
    ks = list(range(0, 80))
    F = cols(dmd.dmd_predict(model, ks, precision=prec), sc.n)
    Fo = O.predict_real(PhiR_o, O.coefficients(ref["lam"], beta_o, ks))
    assert rel(F, Fo) < BAR[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_divergence_free_reconstruction(dmd, prec):
    """Divergence-free input => divergence-free frames (Sec. 4.5)."""
    sc = synth.config0(noise=0.0)
    model = _fit(dmd, sc, 20, prec)
    F = dmd.dmd_predict(model, [0, 7, 99, 100, 250, 500], precision=prec)[:, : sc.n].double().cpu()
    d = synth.div2d(F, sc.N)
    ratio = (d.norm(dim=1) / F.norm(dim=1)).max().item()
    assert ratio < DIV_BAR[prec], ratio


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_sizes_and_odd_rank(dmd, prec):
    """n not a multiple of the tiles (2 * 45^2 = 4050), odd r, short window,
    negative k.  The data have exactly 7 modes -- 3 conjugate pairs and one
    real decaying mode (lambda = 0.93) -- plus noise of 1e-7, so the rank-7
    truncation is well separated from the noise (sigma_1 / sigma_7 = 2.9 and
    sigma_7 / sigma_8 ~ 1e5) and the fit must return the real eigenvalue as a
    real column; eigenvalues and frames within the bar."""
    import math
    sc = synth.linear_modes_scene(45, 2, 3, 33, 77, keep_fp64=True, omega_hi=math.pi, stratified=True)
    extra = synth.make_modes(45, 2, 4, 78)[6].double().numpy()      # a divergence-free real field
    extra *= 0.6 / np.sqrt(np.mean(extra ** 2))
    S64 = sc.extra["S64"] + np.outer(extra, 0.93 ** np.arange(sc.m + 1))
    S64 += 1e-7 * np.random.default_rng(77).standard_normal(S64.shape)
    sc.S[:, : sc.n] = torch.as_tensor(S64.T, dtype=torch.float32)
    r = 7
    ref, PhiR_o, beta_o, _ = oracle_model(sc.X().numpy(), r)
    assert np.sum(np.abs(ref["lam"].imag) == 0) == 1
    model = _fit(dmd, sc, r, prec, oversample=5, power_iters=1)
    lam_g = model.lam()
    _, lam_err = match(lam_g, ref["lam"])
    assert lam_err < BAR[prec], lam_err
    assert np.sum(lam_g.imag == 0) == 1 and np.min(np.abs(lam_g - 0.93)) < 1e-4
    ks = list(range(-3, 40))
    F = cols(dmd.dmd_predict(model, ks, precision=prec), sc.n)
    Fo = O.predict_real(PhiR_o, O.coefficients(ref["lam"], beta_o, ks))
    assert rel(F, Fo) < BAR[prec], rel(F, Fo)


def test_minimum_sizes(dmd):
    """m = 2 snapshots pairs, r = 1."""
    g = np.random.default_rng(1)
    n = 64
    S = torch.zeros((3, 64), dtype=torch.float32)
    x0 = g.standard_normal(n)
    S[0] = torch.as_tensor(x0)
    S[1] = torch.as_tensor(0.9 * x0)
    S[2] = torch.as_tensor(0.81 * x0)
    model = dmd.dmd_fit(S.cuda(), n, 1, oversample=0, power_iters=0)
    torch.cuda.synchronize()
    model.check()
    assert abs(model.lam()[0] - 0.9) < 1e-6
    F = cols(dmd.dmd_predict(model, [0, 3]), n)
    assert rel(F[:, 1], 0.9 ** 3 * x0) < 1e-5


def test_nonfinite_input_is_reported(dmd):
    sc = synth.linear_modes_scene(16, 2, 2, 20, 5)
    S = sc.S.clone()
    S[3, 17] = float("nan")
    model = dmd.dmd_fit(S.cuda(), sc.n, 4, oversample=2, power_iters=1)
    torch.cuda.synchronize()
    assert model.status() == 5   # DMD_ENONFINITE


def test_rank_deficiency_is_reported(dmd):
    sc = synth.linear_modes_scene(16, 2, 2, 30, 6)   # rank 4
    model = dmd.dmd_fit(sc.S.cuda(), sc.n, 10, oversample=2, power_iters=1)
    torch.cuda.synchronize()
    assert model.status() == 4   # DMD_ERANK


def test_host_argument_errors(dmd):
    sc = synth.linear_modes_scene(16, 2, 2, 20, 5)
    with pytest.raises(dmd.DmdError) as e:
        dmd.dmd_fit(sc.S.cuda(), sc.n, 25)          # r > m
    assert e.value.status == 1


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,pairs,m", [(32, 20, 300), (24, 12, 260)])
def test_more_than_256_snapshots(dmd, prec, N, pairs, m):
    """Snapshot counts above 256 (the many-scene workload draws m up to 400):
    the snapshot Gram, the reductions and the sketch products then span more
    than one 256-wide block.  Eigenvalues, mode fields and frames within the bar."""
    import math
    sc = synth.linear_modes_scene(N, 2, pairs, m, 31 + m, sigma_lo=-0.05, omega_hi=math.pi, stratified=True,
                                  noise=1e-5, keep_fp64=False)
    r = 2 * pairs
    ref, PhiR_o, beta_o, _ = oracle_model(sc.X().numpy(), r)
    model = _fit(dmd, sc, r, prec)
    lam_g = model.lam()
    _, lam_err = match(lam_g, ref["lam"])
    assert lam_err < BAR[prec], lam_err
    mp_frob, _ = mode_product_error(cols(model.Phi_R, sc.n), model.beta(), lam_g, PhiR_o, beta_o, ref["lam"])
    assert mp_frob < BAR[prec], mp_frob
