"""dmd_predict_noalloc: frame prediction for callers that cannot allocate GPU
memory (an application that reserves its GPU memory once under its own
allocator and forbids cudaMalloc / cudaFree in its frame loop, or a plug-in
host that gives the library no allocator).  The entry point takes its
workspace from a fixed device array inside the library, so these tests check
that its frames equal those of dmd_predict (which takes a caller-provided
workspace) on two calls in a row: the second call finds the first call's data
in the shared array and must not be affected by it.

This file is named to be collected after every other test file; it passes
both alone in a fresh process (the first call then does the per-device
set-up) and after the rest of the suite."""
import ctypes

import numpy as np
import pytest
import torch

from tests.gpu_util import rel

SCRATCH_BYTES = 16 * 1024 * 1024   # DMD_NOALLOC_SCRATCH_BYTES in include/dmd.h
TOL = {"fp32": 3e-6, "mixed": 3e-5}  # the prediction tolerances of the other parity tests


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


def _model(dmd, n, npairs, nreal, q, seed):
    """Random real-form model: conjugate pairs (2x2 blocks) plus real
    eigenvalues, FP32 modes with a ragged leading dimension."""
    g = np.random.default_rng(seed)
    r = 2 * npairs + nreal
    lam = []
    for _ in range(npairs):
        z = np.exp(g.uniform(-0.03, 0.0) + 1j * g.uniform(0.05, 1.0))
        lam += [z, np.conj(z)]
    lam += list(g.uniform(0.5, 0.99, nreal) * g.choice([-1, 1], nreal))
    lam = np.array(lam, dtype=complex)
    modal = np.zeros(r * (4 + q))
    modal[:r], modal[r:2 * r], modal[2 * r:3 * r] = lam.real, lam.imag, g.standard_normal(r)
    modal[4 * r:] = 0.1 * g.standard_normal(r * q)
    ld = (n + 31) // 32 * 32
    P = torch.zeros((r, ld), dtype=torch.float32)
    P[:, :n] = torch.as_tensor(g.standard_normal((r, n)), dtype=torch.float32)
    return dmd.DmdModel(P.cuda(), torch.as_tensor(modal).cuda(), torch.zeros(8, dtype=torch.int32, device="cuda"),
                        n, r, q)


def _noalloc_call(dmd, model, kt, out, u, prec):
    """One call straight through the C ABI (no Python-side workspace)."""
    d = dmd.PredictDesc(n=model.n, ldPhi=model.ldPhi, ldOut=out.shape[1], r=model.r, K=kt.numel(), q=model.q,
                        steps=0 if u is None else u.shape[0], precision=dmd.PRECISIONS[prec], chunk=0)
    st = dmd.lib().dmd_predict_noalloc(ctypes.byref(d), model.Phi_R.data_ptr(), model.modal.data_ptr(),
                                       kt.data_ptr(), None if u is None else u.data_ptr(), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert st == 0, dmd.lib().dmd_last_error().decode()


@pytest.mark.gpu
@pytest.mark.parametrize("first,second", [("mixed", "fp32"), ("fp32", "mixed")])
def test_noalloc_matches_predict_twice(dmd, first, second):
    """Call 1: a large mixed/FP32 problem (K = 700 frames, the resident-tile
    reconstruction); call 2: a smaller controlled problem in the other
    precision, which reuses the array the first call filled."""
    g = np.random.default_rng(5)
    m1 = _model(dmd, 40000 + 17, 20, 3, 0, 21)
    k1 = torch.as_tensor(np.concatenate([np.arange(600), g.integers(-50, 3000, 100)]).astype(np.int32)).cuda()
    m2 = _model(dmd, 9000 + 5, 6, 2, 2, 22)
    steps = 80
    u2 = torch.as_tensor(g.standard_normal((steps, 2)), dtype=torch.float32).cuda()
    k2 = torch.as_tensor(g.integers(0, steps + 1, 90).astype(np.int32)).cuda()
    for model, kt, u, prec in [(m1, k1, None, first), (m2, k2, u2, second)]:
        ref = dmd.dmd_predict(model, kt, u=u, precision=prec)
        out = torch.full_like(ref, float("nan"))
        _noalloc_call(dmd, model, kt, out, u, prec)
        torch.cuda.synchronize()
        n = model.n
        a = out[:, :n].double().cpu().numpy()
        b = ref[:, :n].double().cpu().numpy()
        assert np.isfinite(a).all()
        assert rel(a, b) < TOL[prec], (prec, rel(a, b))


@pytest.mark.gpu
def test_noalloc_repeated_calls_are_stable(dmd):
    """The same call twice in a row gives the same frames (each call clears
    the part of the array it uses)."""
    model = _model(dmd, 20000 + 3, 10, 1, 0, 23)
    kt = torch.arange(0, 300, dtype=torch.int32, device="cuda")
    ref = dmd.dmd_predict(model, kt, precision="mixed")
    outs = []
    for _ in range(2):
        out = torch.empty_like(ref)
        _noalloc_call(dmd, model, kt, out, None, "mixed")
        outs.append(out)
    torch.cuda.synchronize()
    for out in outs:
        assert rel(out[:, :model.n].double().cpu().numpy(), ref[:, :model.n].double().cpu().numpy()) < TOL["mixed"]


def test_noalloc_rejects_problems_beyond_the_array(dmd):
    """A problem whose forward workspace exceeds the fixed array is refused on
    the host with DMD_EINVAL and a message that names the sizes (no GPU work)."""
    d = dmd.PredictDesc(n=1000, ldPhi=1024, ldOut=1024, r=256, K=SCRATCH_BYTES // (256 * 8) + 1, q=0, steps=0,
                        precision=0, chunk=0)
    st = dmd.lib().dmd_predict_noalloc(ctypes.byref(d), None, None, None, None, None, None)
    assert st == 1
    msg = dmd.lib().dmd_last_error().decode()
    assert "scratch" in msg and str(SCRATCH_BYTES) in msg
