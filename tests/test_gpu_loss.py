"""Streamed per-frame loss and its gradient (the adjoint of the prediction,
Sec. 7.2) through the C ABI, against the FP64 oracle on the same model.

In the mixed form the frames never reach memory: the loss alone comes from
the reconstruction kernel's loss epilogue, the loss with its gradient from the
kernel that recomputes 128-row x 128-frame tiles, forms G = w rho'(x - t) in
its epilogue and accumulates dC^T = G^T Phi_R in tensor memory.  The FP32 form
recomputes stored chunks.  Both are compared with the oracle's loss
(frame_loss) and its gradient (Phi_R^T frame_loss_grad, then the closed-form
adjoint predict_adjoint), for the quadratic and the Huber loss."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

BAR = {"fp32": 1e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


def _model(dmd, n, npairs, nreal, seed):
    """A random real-form model: |lambda| near 1, Phi_R and beta Gaussian."""
    g = np.random.default_rng(seed)
    r = 2 * npairs + nreal
    lam = []
    for _ in range(npairs):
        z = np.exp(g.uniform(-0.01, 0.0) + 1j * g.uniform(0.05, 3.0))
        lam += [z, np.conj(z)]
    lam += list(g.uniform(0.9, 0.999, nreal) * g.choice([-1, 1], nreal))
    lam = np.array(lam, dtype=complex)
    ld = (n + 31) // 32 * 32
    P = torch.zeros((r, ld), dtype=torch.float32)
    P[:, :n] = torch.randn((r, n), generator=torch.Generator().manual_seed(seed), dtype=torch.float32)
    beta = g.standard_normal(r)
    modal = np.zeros(4 * r)
    modal[:r], modal[r:2 * r], modal[2 * r:3 * r] = lam.real, lam.imag, beta
    model = dmd.DmdModel(P.cuda(), torch.as_tensor(modal).cuda(), torch.zeros(8, dtype=torch.int32, device="cuda"),
                         n, r, 0)
    return model, P[:, :n].double().numpy().T, lam, beta


def _check(dmd, model, PhiR, lam, beta, ks, prec, kind, seed):
    n, r = model.n, model.r
    g = np.random.default_rng(seed)
    F = O.predict_real(PhiR, O.coefficients(lam, beta, ks))
    tgt = torch.zeros(model.ldPhi, dtype=torch.float32)
    tgt[:n] = torch.as_tensor(F[:, len(ks) // 2] + 0.3 * g.standard_normal(n) * F.std(), dtype=torch.float32)
    tgt64 = tgt[:n].double().numpy()
    w = g.uniform(0.0, 1.0, len(ks))
    delta = 0.5 * float(np.sqrt(np.mean((F - tgt64[:, None]) ** 2))) if kind == "huber" else 0.0
    Lo = O.frame_loss(F, tgt64, w, kind, delta)
    dC = PhiR.T @ O.frame_loss_grad(F, tgt64, w, kind, delta)
    dlr, dli, db = O.predict_adjoint(lam, beta, ks, dC)
    wt = torch.as_tensor(w).cuda()
    l_only, _, _ = dmd.dmd_predict_loss(model, ks, tgt.cuda(), wt, precision=prec, loss=kind, delta=delta)
    l_grad, dmodal, _ = dmd.dmd_predict_loss(model, ks, tgt.cuda(), wt, want_grad=True, precision=prec, loss=kind,
                                             delta=delta)
    dm = dmodal.cpu().numpy()
    errs = dict(loss=abs(l_only.item() - Lo) / Lo, loss_grad_path=abs(l_grad.item() - Lo) / Lo,
                beta=rel(dm[2 * r:3 * r], db), lam_re=rel(dm[:r], dlr), lam_im=rel(dm[r:2 * r], dli))
    print(f"[{prec} {kind} n={n} r={r} K={len(ks)}] " + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v < BAR[prec], (k, v)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("kind", ["quadratic", "huber"])
def test_streamed_loss_and_gradient_match_oracle(dmd, prec, kind):
    """Ragged rows (4007), an odd rank with a real mode (r = 9), 300 frames
    (two full 128-frame groups and a ragged third), negative k."""
    model, PhiR, lam, beta = _model(dmd, 4007, 4, 1, 21)
    ks = list(range(-5, 295))
    _check(dmd, model, PhiR, lam, beta, ks, prec, kind, 5)


@pytest.mark.parametrize("kind", ["quadratic", "huber"])
def test_fused_loss_many_tiles(dmd, kind):
    """The mixed-form fused kernels at r = 150 (all ten K-slices of the
    coefficient operand, the full tensor-memory layout) on 700,001 rows: every
    CTA walks more than 32 row tiles, so the gradient's tensor-memory
    accumulator is drained into the FP64 partials several times per frame
    group; 300 frames make three groups, the last one ragged."""
    model, PhiR, lam, beta = _model(dmd, 700_001, 75, 0, 22)
    ks = list(range(300))
    _check(dmd, model, PhiR, lam, beta, ks, "mixed", kind, 6)
    # none of the tensor-core kernels' bounded waits ran out
    words = dmd.async_status()
    assert words[0] == 0, words


def test_loss_options_are_checked(dmd):
    model, PhiR, lam, beta = _model(dmd, 1000, 2, 0, 23)
    tgt = torch.zeros(model.ldPhi, dtype=torch.float32, device="cuda")
    w = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(dmd.DmdError) as e:
        dmd.dmd_predict_loss(model, [0, 1, 2, 3], tgt, w, precision="mixed", loss="huber", delta=0.0)
    assert e.value.status == 1
