"""Component parity through the C ABI: Philox, tall products, reductions,
coefficients / reconstruction and the adjoint, each against the FP64 oracle
or the plain definition on the same seeded inputs."""
import numpy as np
import pytest
import torch

from oracle import dmd_oracle as O
from oracle import philox
from tests.gpu_util import cols, rel

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "mixed"]
TOL = {"fp32": 2e-6, "mixed": 2e-5}


@pytest.fixture(scope="module")
def dmd():
    from paper_2502_05339_gb300 import build_lib
    build_lib.build()
    from paper_2502_05339_gb300 import dmd as m
    m.lib()
    return m


def test_philox_bit_exact(dmd):
    """Device Philox4x32-10 equals the oracle's restatement of the published definition."""
    for sid, key in [(0, 0), (0x0D3D0001, 1234), (7, 0xFFFFFFFFFFFFFFFF)]:
        out = dmd.dmd_philox_blocks(300, sid, key).cpu().numpy().view(np.uint32)
        for i in list(range(0, 300, 37)) + [299]:
            ref = philox.philox4x32_10((i & 0xFFFFFFFF, i >> 32, sid, 0), (key & 0xFFFFFFFF, key >> 32))
            assert tuple(int(v) for v in out[i]) == ref


def test_sketch_matrix_matches_oracle(dmd):
    for (m, l, seed) in [(57, 13, 99), (200, 160, 1001), (3, 1, 0)]:
        g = dmd.dmd_sketch_matrix(m, l, seed).cpu().numpy().T      # (m, l)
        o = philox.sketch_matrix(m, l, seed)
        np.testing.assert_allclose(g, o, rtol=1e-13, atol=1e-13)


def _tall(n, K, seed, ld=None):
    g = np.random.default_rng(seed)
    ld = ld or (n + 31) // 32 * 32
    A = torch.zeros((K, ld), dtype=torch.float32)
    A[:, :n] = torch.as_tensor(g.standard_normal((K, n)), dtype=torch.float32)
    return A


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,K,N", [(1, 1, 1), (100, 17, 5), (8192 + 37, 100, 64), (70001, 201, 150),
                                   (4096, 20, 257), (12345, 160, 160)])
def test_gemm_tall(dmd, prec, n, K, N):
    A = _tall(n, K, n + K)
    B = np.random.default_rng(N).standard_normal((N, K))
    C, G = dmd.dmd_gemm_tall(A.cuda(), n, torch.as_tensor(B).cuda(), precision=prec, want_gram=True)
    ref = cols(A, n) @ B.T
    assert rel(cols(C, n), ref) < TOL[prec]
    Cg = cols(C, n)
    assert rel(G.cpu().numpy().T, Cg.T @ Cg) < (1e-6 if prec == "fp32" else TOL[prec])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,Ka,N", [(1, 1, 1), (1000, 20, 21), (8192 + 37, 160, 201), (300001, 64, 64),
                                    (65536, 150, 1)])
def test_gemm_tn(dmd, prec, n, Ka, N):
    A = _tall(n, Ka, 3 * n + Ka)
    B = _tall(n, N, 5 * n + N)
    C = dmd.dmd_gemm_tn(A.cuda(), B.cuda(), n, precision=prec)
    ref = cols(A, n).T @ cols(B, n)
    assert rel(C.cpu().numpy().T, ref) < TOL[prec]


@pytest.mark.parametrize("n,Ka", [(1_000_003, 201), (5003, 9), (70_001, 208), (70_001, 209)])
def test_symmetric_gram_fp32(dmd, n, Ka):
    """The snapshot-Gram shape A^T A on the CUDA cores: up to 208 columns one
    CTA forms the whole triangle of its row chunk (201 columns: the 128^3 x 3
    snapshot matrix's m + 1; 9: two column sets; 208: the largest), beyond
    that the tiled kernel (209).  Against the FP64 product at the FP32 bar,
    exactly symmetric, and the same bits on a second call."""
    A = _tall(n, Ka, 11 * n + Ka).cuda()
    C = dmd.dmd_gemm_tn(A, A, n, precision="fp32")
    ref = cols(A.cpu(), n).T @ cols(A.cpu(), n)
    Cn = C.cpu().numpy()
    assert rel(Cn.T, ref) < TOL["fp32"]
    assert np.array_equal(Cn, Cn.T)
    assert torch.equal(C, dmd.dmd_gemm_tn(A, A, n, precision="fp32"))


@pytest.mark.parametrize("prec", PRECS)
def test_gemm_tn_is_deterministic(dmd, prec):
    A = _tall(200003, 40, 1).cuda()
    B = _tall(200003, 30, 2).cuda()
    c1 = dmd.dmd_gemm_tn(A, B, 200003, precision=prec)
    c2 = dmd.dmd_gemm_tn(A, B, 200003, precision=prec)
    assert torch.equal(c1, c2)


@pytest.mark.parametrize("n,K,N", [(300000, 150, 1000), (5000 + 11, 20, 501), (1000, 1, 65), (70001, 200, 1000),
                                   (20011, 256, 700)])
def test_gemm_tall_many_columns(dmd, n, K, N):
    """The reconstruction shape (K frames >> 256 columns: resident-A kernel).
    The cases cover chunk widths 176 (150 modes), 240, 144 and 128 (256
    modes), ring entries of whole chunks and of part chunks with a shorter
    last entry (200 modes: 7 + 6 K-slices), and ragged last chunks."""
    A = _tall(n, K, 7 + n)
    B = np.random.default_rng(N).standard_normal((N, K))
    for prec in PRECS:
        C = dmd.dmd_gemm_tall(A.cuda(), n, torch.as_tensor(B).cuda(), precision=prec)
        assert rel(cols(C, n), cols(A, n) @ B.T) < TOL[prec], prec


def _random_model(n, npairs, nreal, seed, dev="cuda"):
    g = np.random.default_rng(seed)
    r = 2 * npairs + nreal
    lam = []
    for _ in range(npairs):
        z = np.exp(g.uniform(-0.03, 0.0) + 1j * g.uniform(0.05, 1.0))
        lam += [z, np.conj(z)]
    lam += list(g.uniform(0.5, 0.99, nreal) * g.choice([-1, 1], nreal))
    lam = np.array(lam, dtype=complex)
    PhiR = g.standard_normal((n, r))
    beta = g.standard_normal(r)
    modal = np.zeros(4 * r)
    modal[:r], modal[r:2 * r], modal[2 * r:3 * r] = lam.real, lam.imag, beta
    ld = (n + 31) // 32 * 32
    P = torch.zeros((r, ld), dtype=torch.float32)
    P[:, :n] = torch.as_tensor(PhiR.T, dtype=torch.float32)
    from paper_2502_05339_gb300 import dmd as m
    model = m.DmdModel(P.to(dev), torch.as_tensor(modal).to(dev), torch.zeros(8, dtype=torch.int32, device=dev),
                       n, r, 0)
    return model, cols(P, n), lam, beta


@pytest.mark.parametrize("prec", PRECS)
def test_predict_matches_oracle(dmd, prec):
    """Coefficients (FP64 polar lambda^k) + one real GEMM vs the oracle's
    repeated-squaring powers, including negative and extrapolated k."""
    model, PhiR, lam, beta = _random_model(5000 + 13, 7, 3, 11)
    ks = [0, 1, 2, 5, 99, 100, 101, 500, 999, -1, -10, 37]
    F = dmd.dmd_predict(model, ks, precision=prec)
    Fo = O.predict_real(PhiR, O.coefficients(lam, beta, ks))
    assert rel(cols(F, model.n), Fo) < (3e-6 if prec == "fp32" else 3e-5)


@pytest.mark.parametrize("prec", PRECS)
def test_backward_matches_oracle(dmd, prec):
    model, PhiR, lam, beta = _random_model(3000 + 5, 5, 2, 12)
    ks = [0, 3, 10, 50, 200, -4]
    g = np.random.default_rng(3)
    dF = g.standard_normal((model.n, len(ks)))
    ld = model.ldPhi
    dOut = torch.zeros((len(ks), ld), dtype=torch.float32)
    dOut[:, : model.n] = torch.as_tensor(dF.T, dtype=torch.float32)
    dmodal, _ = dmd.dmd_predict_backward(model, ks, dOut.cuda(), precision=prec)
    dC = PhiR.T @ cols(dOut, model.n)
    dlr, dli, db = O.predict_adjoint(lam, beta, ks, dC)
    dm = dmodal.cpu().numpy()
    r = model.r
    t = 1e-5 if prec == "fp32" else 1e-4
    assert rel(dm[2 * r:3 * r], db) < t
    assert rel(dm[:r], dlr) < t
    assert rel(dm[r:2 * r], dli) < t


def test_streamed_loss_matches_oracle(dmd):
    model, PhiR, lam, beta = _random_model(4000 + 7, 4, 1, 13)
    ks = list(range(0, 120))
    g = np.random.default_rng(8)
    tgt = g.standard_normal(model.n)
    w = g.uniform(0, 1, len(ks))
    ld = model.ldPhi
    tg = torch.zeros(ld, dtype=torch.float32)
    tg[: model.n] = torch.as_tensor(tgt, dtype=torch.float32)
    loss, dmodal, _ = dmd.dmd_predict_loss(model, ks, tg.cuda(), torch.as_tensor(w).cuda(), want_grad=True,
                                           chunk=50)
    F = O.predict_real(PhiR, O.coefficients(lam, beta, ks))
    tgt32 = tg[: model.n].double().numpy()
    Lo = 0.5 * float(np.sum(w * np.sum((F - tgt32[:, None]) ** 2, axis=0)))
    assert abs(loss.item() - Lo) / Lo < 1e-5
    dC = PhiR.T @ ((F - tgt32[:, None]) * w[None, :])
    dlr, dli, db = O.predict_adjoint(lam, beta, ks, dC)
    dm = dmodal.cpu().numpy()
    r = model.r
    assert rel(dm[2 * r:3 * r], db) < 1e-4
    assert rel(dm[:r], dlr) < 1e-4


def test_autograd_function(dmd):
    model, PhiR, lam, beta = _random_model(2000 + 3, 3, 1, 14)
    ks = [0, 2, 9, 30]
    modal = model.modal.clone().requires_grad_(True)
    F = dmd.DmdPredict.apply(modal, None, model, ks, "fp32")
    loss = (F[:, : model.n].double() ** 2).sum()
    loss.backward()
    dC = PhiR.T @ (2 * cols(F.detach(), model.n))
    dlr, dli, db = O.predict_adjoint(lam, beta, ks, dC)
    r = model.r
    gm = modal.grad.cpu().numpy()
    assert rel(gm[2 * r:3 * r], db) < 1e-5
    kinds = O.pair_kinds(lam)
    heads = kinds != 2
    assert rel(gm[:r][heads], dlr[heads]) < 1e-5
    assert np.all(gm[:r][kinds == 2] == 0)


@pytest.mark.parametrize("prec,decades", [("fp32", 4.0), ("mixed", 1.5)])
def test_gram_resolves_weak_directions(dmd, prec, decades):
    """The Gram of an ill-conditioned tall matrix keeps every eigen-direction
    to 10%.  FP32: singular values 1 .. 1e-4 (Gram eigenvalues to 1e-8); the
    snapshot Gram of the fit is formed this way and the first CholeskyQR Gram
    of every sketch is derived from it in FP64.  Mixed (BF16x3, measured error
    ~2e-7 of the largest eigenvalue): singular values 1 .. 3e-2, the range of
    the second CholeskyQR Gram, which sees an already orthonormalised basis."""
    g = np.random.default_rng(0)
    n, l = 8192 * 8, 30
    U, _ = np.linalg.qr(g.standard_normal((n, l)))
    V, _ = np.linalg.qr(g.standard_normal((l, l)))
    Y = ((U * np.logspace(0, -decades, l)) @ V.T).astype(np.float32)
    Yt = torch.as_tensor(Y.T).contiguous().cuda()
    Yd = Y.astype(np.float64)
    Gx = Yd.T @ Yd
    w, E = np.linalg.eigh(Gx)
    G = dmd.dmd_gemm_tn(Yt, Yt, n, precision=prec).cpu().numpy().T
    err = np.abs(np.einsum("ij,ik,kj->j", E, G - Gx, E)) / w
    assert err.max() < 0.1, err[:5]
