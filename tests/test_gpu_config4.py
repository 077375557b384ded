"""The large workload: 256^3 x 3 (n = 50,331,648), m = 300 FP32 snapshots
(~60 GB), data as the 128^3 workload, rSVD at r = 150 with oversampling 16 and
one power iteration (mixed form), then 2000 frames streamed into a per-frame
loss and its gradient, the frames recomputed on the tensor cores and never
stored.  The FP64 oracle
cannot decompose a matrix of this size, so the checks are properties that
hold at any size: the reconstruction of the training window and its
divergence (the data are divergence-free up to their noise), and the streamed
loss and gradient against the same quantities from stored frames (block-wise
dmd_predict and dmd_predict_backward)."""
import gc

import numpy as np
import pytest
import torch

from paper_2502_05339_gb300 import synth

pytestmark = pytest.mark.gpu

R, OVERSAMPLE, POWER, FRAMES, CHUNK, SEED = 150, 16, 1, 2000, 50, 1004


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def fitted(dmd):
    sc = synth.config4(device="cuda")
    model, r = _fit(dmd, sc)
    yield sc, model, r
    # hand the ~100 GB back to the device before the next test module
    del sc, model
    gc.collect()
    torch.cuda.empty_cache()


def _fit(dmd, sc):
    # A drawn pair can sit below what the fit resolves (a tiny random
    # amplitude under the noise): the fit then reports DMD_ERANK, and the
    # rank is lowered in steps of 2 (at most 10 below the workload's 150).
    r = R
    while True:
        model = dmd.dmd_fit(sc.S, sc.n, r, oversample=OVERSAMPLE, power_iters=POWER, precision="mixed", seed=SEED)
        torch.cuda.synchronize()
        if model.status() == 0 or r <= R - 10:
            break
        r -= 2
    model.check()
    return model, r


def _rel(a, b):
    return float((a - b).double().norm() / b.double().norm())


def test_config4_window_and_divergence(dmd, fitted):
    sc, model, r = fitted
    n, N = sc.n, sc.N
    ks = [0, 100, 200, 299]
    F = dmd.dmd_predict(model, ks, precision="mixed")
    for j, k in enumerate(ks):
        x, s = F[j, :n], sc.S[k, :n]
        err = _rel(x, s)
        div_x = float(synth.div3d(x.double(), N).norm() / x.double().norm())
        div_s = float(synth.div3d(s.double(), N).norm() / s.double().norm())
        print(f"rank {r}: frame {k}: window rel error {err:.2e}; divergence {div_x:.2e} (data {div_s:.2e})")
        assert err < 1e-2, (k, err)              # nonlinear term 1e-3 and noise 1e-4 are not in the linear model
        # x = s + e: the divergence of the frame is that of the data plus at most
        # ||div|| ||e|| <= 2 sqrt(3) ||e|| (forward differences on the periodic grid)
        assert div_x <= div_s + 2 * np.sqrt(3) * err * (1 + 1e-6), (k, div_x, div_s, err)


def test_config4_streamed_loss_and_gradient(dmd, fitted):
    sc, model, r = fitted
    n = sc.n
    target = sc.S[0].clone()
    w = torch.ones(FRAMES, dtype=torch.float64, device="cuda")
    ks = torch.arange(FRAMES, dtype=torch.int32, device="cuda")
    res = dmd.dmd_predict_loss(model, ks, target, w, want_grad=True, precision="mixed", chunk=CHUNK)
    loss_s, dmodal_s = res[0], res[1]
    # the same loss and gradient from stored frames, 25 at a time (5 GB each)
    loss_b = torch.zeros((), dtype=torch.float64, device="cuda")
    dmodal_b = None
    for a in range(0, FRAMES, 25):
        kb = ks[a:a + 25]
        G = dmd.dmd_predict(model, kb, precision="mixed")
        G[:, :n] -= target[:n]
        for i in range(G.shape[0]):
            loss_b += 0.5 * (G[i, :n].double() ** 2).sum()
        dm, _ = dmd.dmd_predict_backward(model, kb, G, precision="mixed")
        dmodal_b = dm.clone() if dmodal_b is None else dmodal_b + dm
        del G
    torch.cuda.synchronize()
    ls, lb = float(loss_s), float(loss_b)
    e_loss = abs(ls - lb) / abs(lb)
    e_grad = float((dmodal_s[:2 * model.r] - dmodal_b[:2 * model.r]).norm() / dmodal_b[:2 * model.r].norm())
    e_beta = float((dmodal_s[2 * model.r:3 * model.r] - dmodal_b[2 * model.r:3 * model.r]).norm()
                   / dmodal_b[2 * model.r:3 * model.r].norm())
    print(f"streamed loss {ls:.6e} vs stored {lb:.6e} (rel {e_loss:.1e}); gradient lambda rel {e_grad:.1e}, "
          f"beta rel {e_beta:.1e}")
    assert e_loss < 1e-5
    assert e_grad < 1e-4 and e_beta < 1e-4
