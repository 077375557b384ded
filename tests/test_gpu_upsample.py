"""Upsampling evolution on the device (dmd_upsample, Sec. 6.3.1) against the
FP64 oracle's literal recurrence: with a model given to both sides (seeded
real-form modes and eigenvalues), and end to end (each side fits its own
model of the same snapshots) with inputs from a coarse scene prolonged to the
model's grid."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from paper_2502_05339_gb300 import synth
from tests.gpu_util import cols, rel

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "mixed"]
BAR = {"fp32": 1e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


def _seeded_model(dmd, n, npairs, nreal, seed):
    """Real-form model with unit-RMS random modes and eigenvalues |lambda| in
    [0.97, 1], frequencies spread over (0, pi) (FP32 modes, FP64 modal)."""
    g = np.random.default_rng(seed)
    r = 2 * npairs + nreal
    ld = (n + 31) // 32 * 32
    P = torch.zeros((r, ld), dtype=torch.float32)
    P[:, :n] = torch.as_tensor(g.standard_normal((r, n)) / np.sqrt(1.0), dtype=torch.float32)
    lam = np.exp(g.uniform(-0.03, 0, npairs) + 1j * np.sort(g.uniform(0.01, 3.0, npairs)))
    modal = np.zeros(4 * r)
    modal[0:2 * npairs:2], modal[1:2 * npairs:2] = lam.real, lam.real
    modal[r:r + 2 * npairs:2], modal[r + 1:r + 2 * npairs:2] = lam.imag, -lam.imag
    modal[2 * npairs:r] = g.uniform(0.9, 1.0, nreal)
    model = dmd.DmdModel(P.cuda(), torch.as_tensor(modal).cuda(), torch.zeros(8, dtype=torch.int32, device="cuda"),
                         n, r, 0)
    lam_all = modal[:r] + 1j * modal[r:2 * r]
    return model, P[:, :n].double().numpy().T, lam_all


@pytest.mark.parametrize("prec", PRECS)
def test_upsample_seeded_model(dmd, prec):
    n, T = 30_000 + 5, 40
    model, PhiR, lam = _seeded_model(dmd, n, 12, 2, seed=4)
    g = np.random.default_rng(5)
    ld = model.ldPhi
    inp = torch.zeros((T + 1, ld), dtype=torch.float32)
    inp[:, :n] = torch.as_tensor(g.standard_normal((T + 1, n)), dtype=torch.float32)
    thr = 1.0
    out = dmd.dmd_upsample(model, inp.cuda(), thr, precision=prec)
    torch.cuda.synchronize()
    Hg = cols(out, n)
    X = inp[:, :n].double().numpy().T
    Ho = O.upsample(O.from_real_form(PhiR, lam), lam, X[:, 0], X[:, 1:], thr)
    err = rel(Hg, Ho)
    print(f"[{prec}] seeded model: frames rel Frobenius {err:.2e}")
    assert err < BAR[prec], err


@pytest.mark.parametrize("prec", PRECS)
def test_upsample_fitted_model(dmd, prec):
    """Model: the fit of the 2D 64x64 training scene (rank 20).  Inputs: a
    16x16 scene of other modes and frequencies, prolonged x4; H_0 is the first
    training snapshot.  Low-order modes: |Im Omega| < 0.3."""
    sc = synth.config0(device="cuda")
    model = dmd.dmd_fit(sc.S, sc.n, 20, precision=prec, seed=5)
    coarse = synth.linear_modes_scene(16, 2, 4, 60, 31, noise=0.0, device="cuda")
    L = synth.prolong(coarse.S, 16, 2, 4)
    inp = torch.zeros((61, model.ldPhi), dtype=torch.float32, device="cuda")
    inp[0, :sc.n] = sc.S[0, :sc.n]
    inp[1:, :sc.n] = L[1:, :sc.n]
    out = dmd.dmd_upsample(model, inp, 0.3, precision=prec)
    torch.cuda.synchronize()
    model.check()
    Hg = cols(out, sc.n)
    ref = O.exact_dmd(sc.X().cpu().numpy(), 20)
    X = inp[:, :sc.n].double().cpu().numpy().T
    Ho = O.upsample(ref["Phi"], ref["lam"], X[:, 0], X[:, 1:], 0.3)
    err = rel(Hg, Ho)
    low = int(np.sum(np.abs(np.angle(ref["lam"])) < 0.3))
    print(f"[{prec}] fitted model ({low} of 20 modes low-order): frames rel Frobenius {err:.2e}")
    assert 0 < low < 20
    assert err < BAR[prec], err


def test_upsample_threshold_zero_is_prediction(dmd):
    """No low-order mode: the frames are the model's prediction from
    b = Phi^+ H_0, whatever the inputs (cross-check of two device paths)."""
    n, T = 20_000, 12
    model, PhiR, lam = _seeded_model(dmd, n, 6, 1, seed=8)
    g = np.random.default_rng(9)
    inp = torch.zeros((T + 1, model.ldPhi), dtype=torch.float32)
    inp[:, :n] = torch.as_tensor(g.standard_normal((T + 1, n)), dtype=torch.float32)
    out = dmd.dmd_upsample(model, inp.cuda(), 0.0, precision="fp32")
    X = inp[:, :n].double().numpy().T
    Ho = O.upsample(O.from_real_form(PhiR, lam), lam, X[:, 0], np.zeros((n, T)), 0.0)
    assert rel(cols(out, n), Ho) < 1e-5


def test_upsample_reuses_model_gram(dmd):
    """The Gram stored by one call and passed back (gram_given) gives the same
    frames bit for bit."""
    n, T = 20_000, 10
    model, PhiR, lam = _seeded_model(dmd, n, 6, 1, seed=12)
    g = np.random.default_rng(13)
    inp = torch.zeros((T + 1, model.ldPhi), dtype=torch.float32)
    inp[:, :n] = torch.as_tensor(g.standard_normal((T + 1, n)), dtype=torch.float32)
    inp = inp.cuda()
    gram = torch.zeros((model.r, model.r), dtype=torch.float64, device="cuda")
    a = dmd.dmd_upsample(model, inp, 1.0, precision="mixed", gram=gram).clone()
    b = dmd.dmd_upsample(model, inp, 1.0, precision="mixed", gram=gram, gram_given=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    G = PhiR.T @ PhiR
    assert rel(gram.cpu().numpy(), G) < 1e-6
