"""Temporal editing (Eq. edit_temporal) on the device: the edited eigenvalues
and amplitudes against the oracle's edit of the same fitted model, and the
frames of the edited model against the oracle's prediction."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from paper_2502_05339_gb300 import synth
from tests.gpu_util import cols, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def model(dmd):
    sc = synth.config0()
    mdl = dmd.dmd_fit(sc.S.cuda(), sc.n, 20, oversample=10, power_iters=2, precision="fp32", seed=5)
    torch.cuda.synchronize()
    mdl.check()
    return sc, mdl


@pytest.mark.parametrize("thr,low,high,dt", [
    (0.01, (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 1.0),
    (0.3, (0.5, 1.5, 1.0), (1.5, 0.5, 1.5), 1.0),
    (0.1, (1.0, 0.0, 1.0), (2.0, 1.0, 0.0), 0.5),
    (1e9, (0.25, 2.0, 0.5), (1.0, 1.0, 1.0), 2.0),
])
def test_edit_matches_oracle(dmd, model, thr, low, high, dt):
    sc, mdl = model
    edited = dmd.dmd_edit_modes(mdl, thr, low, high, dt)
    torch.cuda.synchronize()
    r = mdl.r
    lam, beta = mdl.lam(), mdl.beta()
    lam_o, beta_o = O.edit_modes(lam, beta, thr, low, high, dt)
    e = edited.cpu().numpy()
    lam_g = e[:r] + 1j * e[r:2 * r]
    np.testing.assert_allclose(lam_g, lam_o, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(e[2 * r:3 * r], beta_o, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(e[3 * r:4 * r], mdl.sigma())
    ks = [0, 1, 7, 50, -3]
    F = dmd.dmd_predict(mdl, ks, precision="fp32", modal=edited)
    Fo = O.predict_real(cols(mdl.Phi_R, sc.n), O.coefficients(lam_o, beta_o, ks))
    assert rel(cols(F, sc.n), Fo) < 3e-6


def test_edit_rejects_bad_arguments(dmd, model):
    sc, mdl = model
    with pytest.raises(dmd.DmdError):
        dmd.dmd_edit_modes(mdl, 0.01, dt=0.0)
    with pytest.raises(dmd.DmdError):
        dmd.dmd_edit_modes(mdl, -1.0)
