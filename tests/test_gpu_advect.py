"""Density carried by the DMD velocity (dmd_advect_density, Sec. 7.2) against
the FP64 oracle: the same seeded model (divergence-free MAC-grid modes, FP32,
and FP64 eigenvalues) on both sides; the oracle predicts the velocity frames
in FP64 and runs the semi-Lagrangian steps literally.  Grids with
N % 4 == 0 take the four-cells-per-thread kernel (its power-of-two form for
N = 16, 64; the general form for N = 48, 20), the others the one-cell
kernel."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from paper_2502_05339_gb300 import synth
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


def _model(dmd, N, dim, npairs, seed, speed):
    """Real-form model whose modes are synthetic divergence-free MAC fields."""
    g = np.random.default_rng(seed)
    rows = synth.make_modes(N, dim, npairs, seed)                # (2P, n) FP64: Re, Im rows
    n = rows.shape[1]
    r = 2 * npairs
    ld = (n + 31) // 32 * 32
    P = torch.zeros((r, ld), dtype=torch.float32)
    P[:, :n] = rows.to(torch.float32)
    lam = np.exp(g.uniform(-0.02, 0, npairs) + 1j * g.uniform(0.02, 0.4, npairs))
    modal = np.zeros(4 * r)
    modal[0:r:2], modal[1:r:2] = lam.real, lam.real
    modal[r:2 * r:2], modal[r + 1:2 * r:2] = lam.imag, -lam.imag
    modal[2 * r:3 * r] = speed * g.standard_normal(r)
    model = dmd.DmdModel(P.cuda(), torch.as_tensor(modal).cuda(), torch.zeros(8, dtype=torch.int32, device="cuda"),
                         n, r, 0)
    PhiR = P[:, :n].double().numpy().T
    return model, PhiR, modal[:r] + 1j * modal[r:2 * r], modal[2 * r:3 * r]


def _density(N, dim):
    ax = np.arange(N) + 0.5
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    f = 1.0 + 0.5 * np.cos(2 * np.pi * grids[0] / N) * np.sin(4 * np.pi * grids[-1] / N)
    r2 = sum((q - N / 2) ** 2 for q in grids)
    f += 2.0 * np.exp(-r2 / (2 * (N / 8) ** 2))
    return f.ravel().astype(np.float32)


@pytest.mark.parametrize("dim,N,K", [(2, 48, 24), (3, 16, 12), (2, 64, 16), (3, 20, 8), (2, 30, 10), (3, 10, 8)])
@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_advect_matches_oracle(dmd, dim, N, K, prec):
    model, PhiR, lam, beta = _model(dmd, N, dim, 4, seed=21 + dim, speed=0.6)
    rho0 = _density(N, dim)
    dt = 0.5
    out = dmd.dmd_advect_density(model, torch.as_tensor(rho0).cuda(), N, dim, K, dt, precision=prec, chunk=5)
    torch.cuda.synchronize()
    cells = N ** dim
    Rg = out[:, :cells].double().cpu().numpy().T
    frames = O.predict_real(PhiR, O.coefficients(lam, beta, range(K)))
    Ro = O.advect_density(rho0.astype(np.float64), frames, N, dim, dt)
    disp = dt * np.abs(frames).max()
    err = rel(Rg, Ro)
    print(f"[{prec}] {dim}D N={N} K={K}: max displacement {disp:.2f} cells/step, density rel Frobenius {err:.2e}")
    assert disp > 0.3                    # the density really moves
    assert rel(Ro[:, -1], Ro[:, 0]) > 1e-2
    assert err < BAR[prec], err


def test_advect_chunking_is_invisible(dmd):
    """Velocity frames rebuilt in batches of 1, 7 or all K give the same densities bit for bit."""
    N, dim, K = 32, 2, 15
    model, *_ = _model(dmd, N, dim, 3, seed=40, speed=0.5)
    rho0 = torch.as_tensor(_density(N, dim)).cuda()
    outs = [dmd.dmd_advect_density(model, rho0, N, dim, K, 0.4, precision="fp32", chunk=c).clone()
            for c in (1, 7, 0)]
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
