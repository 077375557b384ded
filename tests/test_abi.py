"""The C ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "dmd.h")).read()
    return sorted(set(re.findall(r"^DMD_EXPORT [^(]*?\b(dmd_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libdmd():
    from paper_2502_05339_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("dmd_fit", "dmd_predict", "dmd_predict_backward", "dmd_fit_workspace_bytes",
              "dmd_predict_loss", "dmd_gemm_tall", "dmd_gemm_tn", "dmd_sketch_matrix"):
        assert s in syms


def test_every_declared_symbol_is_exported(libdmd):
    for s in declared_symbols():
        assert hasattr(libdmd, s), s


def test_binding_signatures_cover_header():
    from paper_2502_05339_gb300 import dmd
    assert set(declared_symbols()) == set(dmd.SIGNATURES)


def test_host_side_queries_without_gpu(libdmd):
    """Workspace queries and argument checks are host-only and need no GPU."""
    from paper_2502_05339_gb300 import dmd
    L = dmd.lib()
    d = dmd.FitDesc(n=6291456, ldS=6291456, ldPhi=6291456, m=200, r=150, oversample=10, power_iters=2,
                    q=0, precision=0, seed=1)
    nb = ctypes.c_size_t(0)
    assert L.dmd_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == 0
    assert nb.value > 6291456 * 160 * 4              # the tall basis Q1 at least
    bad = dmd.FitDesc(n=100, ldS=98, ldPhi=100, m=10, r=3, oversample=2, power_iters=1, q=0, precision=0, seed=0)
    assert L.dmd_fit_workspace_bytes(ctypes.byref(bad), ctypes.byref(nb)) == 1   # EINVAL: ldS < n
    assert b"ldS" in L.dmd_last_error()
    bad = dmd.FitDesc(n=100, ldS=100, ldPhi=100, m=10, r=11, oversample=2, power_iters=1, q=0, precision=0, seed=0)
    assert L.dmd_fit_workspace_bytes(ctypes.byref(bad), ctypes.byref(nb)) == 1   # r > m
    p = dmd.PredictDesc(n=100, ldPhi=100, ldOut=100, r=4, K=10, q=0, steps=0, precision=0, chunk=0)
    assert L.dmd_predict_workspace_bytes(ctypes.byref(p), ctypes.byref(nb)) == 0
    # a too-small workspace is refused before any device work
    assert L.dmd_predict(ctypes.byref(p), 16, 16, 16, None, 16, 256, 8, None) == 2   # ENOMEM
    assert L.dmd_async_status(None, 1, None) == 1                                      # EINVAL: no host array
    # the mixed-form loss gradient holds a bf16 hi / lo copy of Phi_R (4 bytes
    # per row and mode, r padded to 16); the loss alone and dmd_predict do not
    p = dmd.PredictDesc(n=6291456, ldPhi=6291456, ldOut=6291456, r=150, K=1000, q=0, steps=0, precision=1, chunk=0)
    nl, ng, npred = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert L.dmd_predict_loss_workspace_bytes(ctypes.byref(p), 0, ctypes.byref(nl)) == 0
    assert L.dmd_predict_loss_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(ng)) == 0
    assert L.dmd_predict_workspace_bytes(ctypes.byref(p), ctypes.byref(npred)) == 0
    split = 6291456 * 160 * 4
    assert ng.value >= split and nl.value < split and npred.value < split


def test_optdmd_rejects_control_and_large_rank():
    """Host-side argument checks of dmd_fit_optdmd (no GPU needed)."""
    import ctypes
    from paper_2502_05339_gb300 import dmd
    L = dmd.lib()
    nb = ctypes.c_size_t(0)
    ok = dmd.FitDesc(n=4096, ldS=4096, ldPhi=4096, m=60, r=20, oversample=10, power_iters=2, q=0, precision=1, seed=0)
    assert L.dmd_fit_optdmd_workspace_bytes(ctypes.byref(ok), ctypes.byref(nb)) == 0 and nb.value > 0
    ctl = dmd.FitDesc(n=4096, ldS=4096, ldPhi=4096, m=60, r=20, oversample=10, power_iters=2, q=2, precision=1, seed=0)
    assert L.dmd_fit_optdmd_workspace_bytes(ctypes.byref(ctl), ctypes.byref(nb)) == 1
    big = dmd.FitDesc(n=4096, ldS=4096, ldPhi=4096, m=400, r=210, oversample=10, power_iters=2, q=0, precision=1,
                      seed=0)
    assert L.dmd_fit_optdmd_workspace_bytes(ctypes.byref(big), ctypes.byref(nb)) == 1


def test_upsample_argument_checks():
    """Host-side checks of dmd_upsample's request (no GPU needed)."""
    import ctypes
    from paper_2502_05339_gb300 import dmd
    L = dmd.lib()
    nb = ctypes.c_size_t(0)

    def desc(**kw):
        base = dict(n=4096, ldPhi=4096, ldIn=4096, ldOut=4096, r=20, T=10, precision=1, gram_given=0,
                    threshold=0.3, dt=1.0)
        base.update(kw)
        return dmd.UpsampleDesc(**base)

    assert L.dmd_upsample_workspace_bytes(ctypes.byref(desc()), ctypes.byref(nb)) == 0 and nb.value > 0
    for bad in (dict(T=0), dict(r=201), dict(ldIn=4094), dict(dt=0.0), dict(threshold=-1.0), dict(gram_given=2),
                dict(ldOut=100)):
        assert L.dmd_upsample_workspace_bytes(ctypes.byref(desc(**bad)), ctypes.byref(nb)) == 1, bad
    d = desc(gram_given=1)
    ws = ctypes.c_void_p(256)
    # gram_given without a gram buffer is refused before anything is launched
    assert L.dmd_upsample(ctypes.byref(d), ws, ws, ws, ws, None, ws, ws, 1 << 30, None) == 1


def test_advect_argument_checks():
    """Host-side checks of dmd_advect_density's request (no GPU needed)."""
    import ctypes
    from paper_2502_05339_gb300 import dmd
    L = dmd.lib()
    nb = ctypes.c_size_t(0)

    def desc(**kw):
        base = dict(ldPhi=2 * 32 * 32, ldRho=32 * 32, N=32, dim=2, r=10, K=5, precision=1, chunk=0, dt=0.5)
        base.update(kw)
        return dmd.AdvectDesc(**base)

    assert L.dmd_advect_workspace_bytes(ctypes.byref(desc()), ctypes.byref(nb)) == 0 and nb.value > 0
    for bad in (dict(dim=4), dict(N=1), dict(K=0), dict(r=0), dict(ldRho=1000), dict(ldPhi=2047),
                dict(dt=float("nan")), dict(chunk=-1), dict(dim=3, N=2000, ldPhi=3 * 2000 ** 3, ldRho=2000 ** 3)):
        assert L.dmd_advect_workspace_bytes(ctypes.byref(desc(**bad)), ctypes.byref(nb)) == 1, bad


def test_binding_refuses_short_outputs_and_bad_controls():
    """The C ABI cannot see buffer sizes, so the binding checks them before any
    call: a frame buffer with fewer than K frames or n rows, a missing,
    misshaped or host-resident control sequence, and a short modal buffer are
    refused on the host (no library call, no GPU needed)."""
    import torch
    from paper_2502_05339_gb300 import dmd
    n, r = 100, 4
    model = dmd.DmdModel(torch.zeros((r, 128)), torch.zeros(4 * r, dtype=torch.float64),
                         torch.zeros(8, dtype=torch.int32), n, r, 0)
    ks = list(range(10))
    with pytest.raises(ValueError):
        dmd.dmd_predict(model, ks, out=torch.zeros((9, 128)))            # 9 < K frames
    with pytest.raises(ValueError):
        dmd.dmd_predict(model, ks, out=torch.zeros((10, 96)))            # 96 < n rows
    with pytest.raises(ValueError):
        dmd.dmd_predict_noalloc(model, ks, torch.zeros((10, 64)))
    with pytest.raises(ValueError):
        dmd.dmd_predict_backward(model, ks, torch.zeros((3, 128)))
    with pytest.raises(ValueError):
        dmd.dmd_predict(model, ks, u=torch.zeros((5, 2)), out=torch.zeros((10, 128)))   # no control inputs
    ctl = dmd.DmdModel(torch.zeros((r, 128)), torch.zeros(6 * r, dtype=torch.float64),
                       torch.zeros(8, dtype=torch.int32), n, r, 2)
    with pytest.raises(ValueError):
        dmd.dmd_predict(ctl, ks, out=torch.zeros((10, 128)))             # q > 0 needs u
    with pytest.raises(ValueError):
        dmd.dmd_predict(ctl, ks, u=torch.zeros((5, 3)), out=torch.zeros((10, 128)))   # q mismatch
    with pytest.raises(TypeError):
        dmd.dmd_predict_noalloc(ctl, ks, torch.zeros((10, 128)), u=torch.zeros((5, 2)))   # host u
    with pytest.raises(ValueError):
        dmd.dmd_predict(model, ks, out=torch.zeros((10, 128)), modal=torch.zeros(3, dtype=torch.float64))
