"""Parity at the full 128^3 x 3 size (n = 6,291,456 values per snapshot,
m = 200, rank 150, oversampling 10, two power iterations, frames k = 0..999):
the launch configuration the benchmark times, in both precision forms.

The FP64 oracle cannot decompose the 6.3M x 200 snapshot matrix directly in a
test, so it evaluates the same exact-DMD definition from inner products: the
snapshot Gram S^T S is formed on the host in FP64 (column blocks of the same
FP32 snapshots the GPU sees), and modes and frames are evaluated at 4,098
sampled rows (random rows plus the first and the last, ragged-tail, row)."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from paper_2502_05339_gb300 import synth
from tests.gpu_util import eig_frob, match, mode_product_error, rel

pytestmark = pytest.mark.gpu

BAR = {"fp32": 1e-5, "mixed": 1e-4}
R, OVERSAMPLE, POWER, FRAMES, SEED = 150, 10, 2, 1000, 1001


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def gram_rows():
    sc = synth.config1(seed=SEED, device="cuda")
    S, n = sc.S, sc.n
    mp1 = S.shape[0]
    Wg = np.zeros((mp1, mp1))
    step = 1 << 20
    for a in range(0, n, step):
        blk = S[:, a:min(n, a + step)].cpu().numpy().astype(np.float64)
        Wg += blk @ blk.T
    g = np.random.default_rng(7)
    rows = np.unique(np.concatenate([[0, n - 1], g.choice(n, 4096, replace=False)]))
    Srows = S[:, torch.as_tensor(rows, device=S.device)].cpu().numpy().astype(np.float64).T   # rows x (m+1)
    return sc, Wg, rows, Srows


@pytest.fixture(scope="module")
def scene_and_oracle(gram_rows):
    sc, Wg, rows, Srows = gram_rows
    ref = O.exact_dmd_from_gram(Wg, R, Srows[:, 1:])
    PhiR, beta, kinds = O.to_real_form(ref["Phi_rows"], ref["lam"], ref["b"])
    frames = O.predict_real(PhiR, O.coefficients(ref["lam"], beta, range(FRAMES)))
    return sc, rows, ref, PhiR, beta, frames


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_config1_full_size(dmd, scene_and_oracle, prec):
    sc, rows, ref, PhiR_o, beta_o, frames_o = scene_and_oracle
    model = dmd.dmd_fit(sc.S, sc.n, R, oversample=OVERSAMPLE, power_iters=POWER, precision=prec, seed=SEED)
    model.check()
    out = dmd.dmd_predict(model, torch.arange(FRAMES, dtype=torch.int32, device="cuda"), precision=prec)
    ridx = torch.as_tensor(rows, device=out.device)
    frames_g = out[:, ridx].double().cpu().numpy().T                 # rows x frames
    PhiR_g = model.Phi_R[:, ridx].double().cpu().numpy().T
    del out
    torch.cuda.empty_cache()
    lam_g, beta_g = model.lam(), model.beta()
    # eigenvalues (matched), scale-free mode fields phi_j b_j and the frames at the sampled rows
    _, worst = match(lam_g, ref["lam"])
    frob, per_mode = mode_product_error(PhiR_g, beta_g, lam_g, PhiR_o, beta_o, ref["lam"])
    err = rel(frames_g, frames_o)
    print(f"[{prec}] eigenvalues max rel {worst:.3e}; mode products rel Frobenius {frob:.3e} "
          f"(worst mode {per_mode.max():.3e}); frames rel Frobenius {err:.3e}")
    assert worst < BAR[prec], ("eigenvalues", worst)
    assert frob < BAR[prec], ("mode products", frob)
    assert err < BAR[prec], ("frames", err)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_config1_optdmd_full_size(dmd, gram_rows, prec):
    """OptDMD (Sec. 4.2) at the same size: eigenvalues, mode fields phi_j b_j
    and frames at the sampled rows against the oracle's inner-product route."""
    sc, Wg, rows, Srows = gram_rows
    ref = O.optdmd_from_gram(Wg, R, Srows[:, :-1])
    PhiR_o, beta_o, _ = O.to_real_form(ref["Phi_rows"], ref["lam"], ref["b"])
    frames_o = O.predict_real(PhiR_o, O.coefficients(ref["lam"], beta_o, range(FRAMES)))
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    model = dmd.dmd_fit_optdmd(sc.S, sc.n, R, oversample=OVERSAMPLE, power_iters=POWER, precision=prec,
                               seed=SEED, stats=stats)
    model.check()
    out = dmd.dmd_predict(model, torch.arange(FRAMES, dtype=torch.int32, device="cuda"), precision=prec)
    ridx = torch.as_tensor(rows, device=out.device)
    frames_g = out[:, ridx].double().cpu().numpy().T
    PhiR_g = model.Phi_R[:, ridx].double().cpu().numpy().T
    del out
    torch.cuda.empty_cache()
    lam_g, beta_g = model.lam(), model.beta()
    _, worst = match(lam_g, ref["lam"])
    lam_frob = eig_frob(lam_g, ref["lam"])
    frob, per_mode = mode_product_error(PhiR_g, beta_g, lam_g, PhiR_o, beta_o, ref["lam"])
    err = rel(frames_g, frames_o)
    f0, f, evals, acc = stats.cpu().tolist()
    print(f"[{prec}] OptDMD objective {f0:.6e} -> {f:.6e} ({evals:.0f} evaluations, {acc:.0f} accepted); oracle "
          f"{ref['f0']:.6e} -> {ref['f']:.6e} ({ref['iters']} iterations); eigenvalues rel Frobenius "
          f"{lam_frob:.3e} (max rel {worst:.3e}); mode products rel Frobenius {frob:.3e} "
          f"(worst mode {per_mode.max():.3e}); frames {err:.3e}")
    # The bar is the relative Frobenius error of each result; for OptDMD's
    # eigenvalues that is the matched eigenvalue vector, not each value.  The
    # weakest modes' eigenvalues are the most sensitive part of the fit (the
    # objective is flattest along them): the FP64 oracle's own OptDMD of this
    # recipe (16^3 x 3 grid) moves its worst single eigenvalue by 2.8e-5 when
    # the snapshots are perturbed by a relative 1e-7 (FP32 rounding) and by
    # 8.5e-4 at 7.6e-6 (the BF16x3 split's rounding), while its eigenvalue
    # vector moves by 1.7e-7 and 5.2e-6.  A per-value bar of 1e-5 / 1e-4 is
    # therefore below what the data's rounding allows; the vector's is not.
    assert lam_frob < BAR[prec], ("eigenvalues", lam_frob)
    assert frob < BAR[prec], ("mode products", frob)
    assert err < BAR[prec], ("frames", err)
