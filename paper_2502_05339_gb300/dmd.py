"""Thin Python binding of libdmd (argument marshalling only).

Every step of the DMD path runs inside libdmd's CUDA kernels; this module only
checks tensor shapes, allocates outputs and workspace through PyTorch's
caching allocator, and passes raw device pointers plus the current CUDA
stream across the C ABI (include/dmd.h).  If the library has not been built
it raises -- there is no CPU or PyTorch fallback.

Column-major matrices are torch tensors of shape (cols, ld): row c of the
tensor is column c of the matrix.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdmd.so")

DMD_FP32, DMD_MIXED_BF16X3 = 0, 1
PRECISIONS = {"fp32": DMD_FP32, "mixed": DMD_MIXED_BF16X3, "bf16x3": DMD_MIXED_BF16X3}
STATUS = {0: "DMD_OK", 1: "DMD_EINVAL", 2: "DMD_ENOMEM", 3: "DMD_ENUMERIC", 4: "DMD_ERANK",
          5: "DMD_ENONFINITE", 6: "DMD_ETIMEOUT", 7: "DMD_ECUDA"}
INFO_WORDS = 8


class DmdError(RuntimeError):
    def __init__(self, what: str, status: int, message: str = ""):
        super().__init__(f"{what}: {STATUS.get(status, status)} {message}".strip())
        self.status = status


class FitDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ldS", ctypes.c_int64), ("ldPhi", ctypes.c_int64),
                ("m", ctypes.c_int32), ("r", ctypes.c_int32), ("oversample", ctypes.c_int32),
                ("power_iters", ctypes.c_int32), ("q", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class OptDmdOpts(ctypes.Structure):
    _fields_ = [("max_evals", ctypes.c_int32), ("reserved", ctypes.c_int32), ("tol", ctypes.c_double),
                ("mu0", ctypes.c_double)]


class UpsampleDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ldPhi", ctypes.c_int64), ("ldIn", ctypes.c_int64), ("ldOut", ctypes.c_int64),
                ("r", ctypes.c_int32), ("T", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("gram_given", ctypes.c_int32), ("threshold", ctypes.c_double), ("dt", ctypes.c_double)]


class AdvectDesc(ctypes.Structure):
    _fields_ = [("ldPhi", ctypes.c_int64), ("ldRho", ctypes.c_int64), ("N", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("r", ctypes.c_int32), ("K", ctypes.c_int32), ("precision", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("dt", ctypes.c_double)]


class LossOpts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("delta", ctypes.c_double)]


LOSS_KINDS = {"quadratic": 0, "huber": 1}


class PredictDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ldPhi", ctypes.c_int64), ("ldOut", ctypes.c_int64),
                ("r", ctypes.c_int32), ("K", ctypes.c_int32), ("q", ctypes.c_int32),
                ("steps", ctypes.c_int32), ("precision", ctypes.c_int32), ("chunk", ctypes.c_int32)]


_P = ctypes.c_void_p
_SZ = ctypes.POINTER(ctypes.c_size_t)


class Scene(ctypes.Structure):
    _fields_ = [("fit", FitDesc), ("S", _P), ("Phi_R", _P), ("modal", _P), ("info", _P), ("K", ctypes.c_int32),
                ("k", _P), ("out", _P), ("ldOut", ctypes.c_int64)]

SIGNATURES = {
    "dmd_last_error": (ctypes.c_char_p, []),
    "dmd_version": (ctypes.c_char_p, []),
    "dmd_launch_count": (ctypes.c_uint64, []),
    "dmd_async_status": (ctypes.c_int32, [_P, ctypes.c_int32, _P]),
    "dmd_fit_workspace_bytes": (ctypes.c_int32, [ctypes.POINTER(FitDesc), _SZ]),
    "dmd_fit": (ctypes.c_int32, [ctypes.POINTER(FitDesc), _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "dmd_advect_workspace_bytes": (ctypes.c_int32, [ctypes.POINTER(AdvectDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "dmd_advect_density": (ctypes.c_int32, [ctypes.POINTER(AdvectDesc), _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "dmd_upsample_workspace_bytes": (ctypes.c_int32, [ctypes.POINTER(UpsampleDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "dmd_upsample": (ctypes.c_int32, [ctypes.POINTER(UpsampleDesc), _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t,
                                      _P]),
    "dmd_fit_optdmd_workspace_bytes": (ctypes.c_int32, [ctypes.POINTER(FitDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "dmd_fit_optdmd": (ctypes.c_int32, [ctypes.POINTER(FitDesc), ctypes.POINTER(OptDmdOpts), _P, _P, _P, _P, _P,
                                        _P, _P, ctypes.c_size_t, _P]),
    "dmd_predict_workspace_bytes": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), _SZ]),
    "dmd_predict_loss_workspace_bytes": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), ctypes.c_int32, _SZ]),
    "dmd_predict": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "dmd_predict_noalloc": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), _P, _P, _P, _P, _P, _P]),
    "dmd_predict_backward": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), _P, _P, _P, _P, _P, _P, _P, _P,
                                              ctypes.c_size_t, _P]),
    "dmd_predict_loss": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), _P, _P, _P, _P, _P, _P,
                                          ctypes.POINTER(LossOpts), ctypes.c_int32, _P, _P, _P, _P, ctypes.c_size_t,
                                          _P]),
    "dmd_edit_modes": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_double, _P, _P,
                                        ctypes.c_double, _P]),
    "dmd_autotune_predict": (ctypes.c_int32, [ctypes.POINTER(PredictDesc), _P, _P, _P, _P, _P, ctypes.c_size_t, _P,
                                              _P]),
    "dmd_batch_workspace_bytes": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(Scene), ctypes.c_int32, _SZ]),
    "dmd_fit_predict_batch": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(Scene), ctypes.c_int32, _P,
                                               ctypes.c_size_t, _P]),
    "dmd_sketch_matrix": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P]),
    "dmd_philox_blocks": (ctypes.c_int32, [ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, _P, _P]),
    "dmd_gemm_tall_workspace_bytes": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                       ctypes.c_int32, _SZ]),
    "dmd_gemm_tall": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P,
                                       ctypes.c_int64, _P, _P, ctypes.c_int64, _P, _P, ctypes.c_size_t, _P]),
    "dmd_gemm_tn_workspace_bytes": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                     ctypes.c_int32, _SZ]),
    "dmd_gemm_tn": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P,
                                     ctypes.c_int64, _P, ctypes.c_int64, _P, _P, ctypes.c_size_t, _P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libdmd.so (built by build_lib.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdmd is not built ({LIB_PATH} missing): run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise DmdError(what, status, lib().dmd_last_error().decode())


def async_status(device=None, clear: bool = True) -> list[int]:
    """The asynchronous status words of the current (or given) device after
    the work queued on its current stream: [0] is DMD_ETIMEOUT if a bounded
    wait of a call without an info argument ran out, [4] its site."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    words = (ctypes.c_int32 * INFO_WORDS)()
    with torch.cuda.device(dev):
        _check(lib().dmd_async_status(ctypes.cast(words, ctypes.c_void_p), 1 if clear else 0, _stream(dev)),
               "dmd_async_status")
    return list(words)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _need_cuda(t: torch.Tensor, name: str, dtype):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def round_up(x: int, a: int) -> int:
    return (x + a - 1) // a * a


def modal_doubles(r: int, q: int) -> int:
    return r * (4 + q)


@dataclass
class DmdModel:
    """Device-resident fit result (real 2x2-block layout of include/dmd.h)."""
    Phi_R: torch.Tensor   # (r, ldPhi) float32 = column-major n x r
    modal: torch.Tensor   # (r * (4 + q),) float64
    info: torch.Tensor    # (8,) int32 status words
    n: int
    r: int
    q: int = 0

    @property
    def ldPhi(self) -> int:
        return self.Phi_R.shape[1]

    def status(self) -> int:
        return int(self.info[0].item())

    def lam(self) -> np.ndarray:
        m = self.modal.cpu().numpy()
        return m[: self.r] + 1j * m[self.r: 2 * self.r]

    def beta(self) -> np.ndarray:
        return self.modal[2 * self.r: 3 * self.r].cpu().numpy()

    def sigma(self) -> np.ndarray:
        return self.modal[3 * self.r: 4 * self.r].cpu().numpy()

    def G(self) -> np.ndarray:
        return self.modal[4 * self.r:].cpu().numpy().reshape(self.q, self.r).T

    def check(self):
        s = self.status()
        if s != 0:
            raise DmdError("dmd_fit (device)", s, f"info={self.info.cpu().tolist()}")


def dmd_fit(S: torch.Tensor, n: int, r: int, *, oversample: int = 10, power_iters: int = 2,
            precision="fp32", seed: int = 0, Ups: torch.Tensor | None = None,
            Omega: torch.Tensor | None = None) -> DmdModel:
    """Fit the DMD (DMDc with Ups) model of S = [x_0..x_m] (tensor (m+1, ldS) float32)."""
    _need_cuda(S, "S", torch.float32)
    m = S.shape[0] - 1
    ldS = S.shape[1]
    q = 0
    if Ups is not None:           # tensor (m, q): column k of the q x m input matrix is Ups[k]
        _need_cuda(Ups, "Ups", torch.float32)
        q = Ups.shape[1]
    if Omega is not None:
        _need_cuda(Omega, "Omega", torch.float64)
    dev = S.device
    ldPhi = round_up(n, 32)
    d = FitDesc(n=n, ldS=ldS, ldPhi=ldPhi, m=m, r=r, oversample=oversample, power_iters=power_iters,
                q=q, precision=_prec(precision), seed=seed)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)), "dmd_fit_workspace_bytes")
    ws = _workspace(nb.value, dev)
    Phi = torch.empty((r, ldPhi), dtype=torch.float32, device=dev)
    if ldPhi > n:
        Phi[:, n:].zero_()
    modal = torch.empty(modal_doubles(r, q), dtype=torch.float64, device=dev)
    info = torch.zeros(INFO_WORDS, dtype=torch.int32, device=dev)
    _check(lib().dmd_fit(ctypes.byref(d), _ptr(S), _ptr(Ups), _ptr(Omega), _ptr(Phi), _ptr(modal), _ptr(info),
                         _ptr(ws), ws.numel(), _stream(dev)), "dmd_fit")
    return DmdModel(Phi, modal, info, n, r, q)


def dmd_fit_optdmd(S: torch.Tensor, n: int, r: int, *, oversample: int = 10, power_iters: int = 2,
                   precision="fp32", seed: int = 0, Omega: torch.Tensor | None = None, max_evals: int = 0,
                   tol: float = 0.0, mu0: float = 0.0, stats: torch.Tensor | None = None) -> DmdModel:
    """OptDMD fit (Sec. 4.2) of S = [x_0..x_m] (tensor (m+1, ldS) float32), started
    from the exact-DMD eigenvalues of the same randomized SVD.  `stats` (4 float64
    on the device, optional) receives the objective at the start, the final
    objective, the evaluations and the accepted steps."""
    _need_cuda(S, "S", torch.float32)
    m = S.shape[0] - 1
    ldS = S.shape[1]
    if Omega is not None:
        _need_cuda(Omega, "Omega", torch.float64)
    if stats is not None:
        _need_cuda(stats, "stats", torch.float64)
    dev = S.device
    ldPhi = round_up(n, 32)
    d = FitDesc(n=n, ldS=ldS, ldPhi=ldPhi, m=m, r=r, oversample=oversample, power_iters=power_iters,
                q=0, precision=_prec(precision), seed=seed)
    o = OptDmdOpts(max_evals=max_evals, reserved=0, tol=tol, mu0=mu0)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_fit_optdmd_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)), "dmd_fit_optdmd_workspace_bytes")
    ws = _workspace(nb.value, dev)
    Phi = torch.empty((r, ldPhi), dtype=torch.float32, device=dev)
    if ldPhi > n:
        Phi[:, n:].zero_()
    modal = torch.empty(modal_doubles(r, 0), dtype=torch.float64, device=dev)
    info = torch.zeros(INFO_WORDS, dtype=torch.int32, device=dev)
    _check(lib().dmd_fit_optdmd(ctypes.byref(d), ctypes.byref(o), _ptr(S), _ptr(Omega), _ptr(Phi), _ptr(modal),
                                _ptr(info), _ptr(stats), _ptr(ws), ws.numel(), _stream(dev)), "dmd_fit_optdmd")
    return DmdModel(Phi, modal, info, n, r, 0)


def dmd_upsample(model: DmdModel, inputs: torch.Tensor, threshold: float, *, dt: float = 1.0, precision="fp32",
                 out: torch.Tensor | None = None, info: torch.Tensor | None = None,
                 gram: torch.Tensor | None = None, gram_given: bool = False) -> torch.Tensor:
    """Upsampling evolution (Sec. 6.3.1): `inputs` (T+1, ldIn) float32 holds H_0
    and L_1..L_T on the model's grid; returns H_1..H_T as (T, ldOut) float32.
    Modes with |Im log(lambda)| / dt < threshold follow the inputs, the others
    evolve from H_0.  `gram` (r x r float64 on the device) receives the model's
    Gram Phi_R^T Phi_R, or supplies it when gram_given."""
    _need_cuda(inputs, "inputs", torch.float32)
    if model.q != 0:
        raise ValueError("dmd_upsample: the model must have no control inputs")
    dev = model.Phi_R.device
    T = inputs.shape[0] - 1
    ldOut = round_up(model.n, 32)
    if out is None:
        out = torch.empty((T, ldOut), dtype=torch.float32, device=dev)
    _need_cuda(out, "out", torch.float32)
    if info is None:
        info = torch.zeros(INFO_WORDS, dtype=torch.int32, device=dev)
    if gram is not None:
        _need_cuda(gram, "gram", torch.float64)
    d = UpsampleDesc(n=model.n, ldPhi=model.ldPhi, ldIn=inputs.shape[1], ldOut=out.shape[1], r=model.r, T=T,
                     precision=_prec(precision), gram_given=1 if gram_given else 0, threshold=threshold, dt=dt)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_upsample_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)), "dmd_upsample_workspace_bytes")
    ws = _workspace(nb.value, dev)
    _check(lib().dmd_upsample(ctypes.byref(d), _ptr(model.Phi_R), _ptr(model.modal), _ptr(inputs), _ptr(out),
                              _ptr(gram), _ptr(info), _ptr(ws), ws.numel(), _stream(dev)), "dmd_upsample")
    return out


def dmd_advect_density(model: DmdModel, rho0: torch.Tensor, N: int, dim: int, K: int, dt: float, *,
                       precision="fp32", chunk: int = 0, out: torch.Tensor | None = None) -> torch.Tensor:
    """Density advected by the model's velocity frames u_0..u_{K-1} (Sec. 7.2):
    rho0 is the cell-centred density (N^dim float32 on the device); returns
    rho_0..rho_K as a (K+1, ldRho) float32 tensor."""
    _need_cuda(rho0, "rho0", torch.float32)
    if model.q != 0:
        raise ValueError("dmd_advect_density: the model must have no control inputs")
    dev = model.Phi_R.device
    cells = N ** dim
    ldRho = round_up(cells, 32)
    if out is None:
        out = torch.empty((K + 1, ldRho), dtype=torch.float32, device=dev)
    _need_cuda(out, "out", torch.float32)
    d = AdvectDesc(ldPhi=model.ldPhi, ldRho=out.shape[1], N=N, dim=dim, r=model.r, K=K, precision=_prec(precision),
                   chunk=chunk, dt=dt)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_advect_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)), "dmd_advect_workspace_bytes")
    ws = _workspace(nb.value, dev)
    _check(lib().dmd_advect_density(ctypes.byref(d), _ptr(model.Phi_R), _ptr(model.modal), _ptr(rho0), _ptr(out),
                                    _ptr(ws), ws.numel(), _stream(dev)), "dmd_advect_density")
    return out


def _ks_tensor(ks, dev) -> torch.Tensor:
    if isinstance(ks, torch.Tensor):
        t = ks.to(device=dev, dtype=torch.int32).contiguous()
    else:
        t = torch.as_tensor(np.asarray(ks, dtype=np.int32), device=dev)
    return t


def _check_frames(model: DmdModel, K: int, t: torch.Tensor, name: str):
    """A (K, ld) frame tensor must hold K frames of at least n rows: the C ABI
    cannot see a buffer's size, so a short one would be written past its end."""
    if t.dim() != 2 or t.shape[0] < K or t.shape[1] < model.n:
        raise ValueError(f"{name} must have shape (>= {K}, >= {model.n}), got {tuple(t.shape)}")
    _need_cuda(t, name, torch.float32)


def _check_control(model: DmdModel, u: torch.Tensor | None):
    """u (steps, q) float32 on the device: needed exactly when the model has
    control inputs."""
    if model.q == 0:
        if u is not None:
            raise ValueError("u given for a model without control inputs")
        return
    if u is None:
        raise ValueError(f"the model has q = {model.q} control inputs: u (steps, q) is required")
    if u.dim() != 2 or u.shape[1] != model.q:
        raise ValueError(f"u must have shape (steps, {model.q}), got {tuple(u.shape)}")
    _need_cuda(u, "u", torch.float32)


def _check_modal(model: DmdModel, modal: torch.Tensor | None) -> torch.Tensor:
    md = model.modal if modal is None else modal
    if md.numel() < modal_doubles(model.r, model.q):
        raise ValueError(f"modal must hold {modal_doubles(model.r, model.q)} doubles, got {md.numel()}")
    _need_cuda(md, "modal", torch.float64)
    return md


def _pdesc(model: DmdModel, K: int, ldOut: int, precision, steps: int = 0, chunk: int = 0) -> PredictDesc:
    return PredictDesc(n=model.n, ldPhi=model.ldPhi, ldOut=ldOut, r=model.r, K=K, q=model.q, steps=steps,
                       precision=_prec(precision), chunk=chunk)


def _pred_ws(d: PredictDesc, dev) -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_predict_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)), "dmd_predict_workspace_bytes")
    return _workspace(nb.value, dev)


def dmd_predict(model: DmdModel, ks, *, u: torch.Tensor | None = None, precision="fp32",
                out: torch.Tensor | None = None, modal: torch.Tensor | None = None) -> torch.Tensor:
    """Frames x_k = Phi_R C[:, k] (tensor (K, ldOut) float32)."""
    dev = model.Phi_R.device
    kt = _ks_tensor(ks, dev)
    K = kt.numel()
    ldOut = round_up(model.n, 32)
    _check_control(model, u)
    if modal is not None:
        _check_modal(model, modal)
    steps = 0 if u is None else u.shape[0]
    if out is None:
        out = torch.empty((K, ldOut), dtype=torch.float32, device=dev)
    _check_frames(model, K, out, "out")
    ldOut = out.shape[1]
    d = _pdesc(model, K, ldOut, precision, steps)
    ws = _pred_ws(d, dev)
    md = _check_modal(model, modal)
    _check(lib().dmd_predict(ctypes.byref(d), _ptr(model.Phi_R), _ptr(md), _ptr(kt), _ptr(u), _ptr(out),
                             _ptr(ws), ws.numel(), _stream(dev)), "dmd_predict")
    return out


def dmd_predict_noalloc(model: DmdModel, ks, out: torch.Tensor, *, u: torch.Tensor | None = None,
                        precision="fp32", modal: torch.Tensor | None = None) -> torch.Tensor:
    """dmd_predict into a caller-provided `out` (K, ldOut) float32 without any
    workspace: the library uses its fixed device scratch array
    (DMD_NOALLOC_SCRATCH_BYTES) instead of allocating.  `ks` should already be
    an int32 CUDA tensor if the caller must not allocate at all."""
    dev = model.Phi_R.device
    kt = _ks_tensor(ks, dev)
    _check_frames(model, kt.numel(), out, "out")
    _check_control(model, u)
    steps = 0 if u is None else u.shape[0]
    d = _pdesc(model, kt.numel(), out.shape[1], precision, steps)
    md = _check_modal(model, modal)
    _check(lib().dmd_predict_noalloc(ctypes.byref(d), _ptr(model.Phi_R), _ptr(md), _ptr(kt), _ptr(u), _ptr(out),
                                     _stream(dev)), "dmd_predict_noalloc")
    return out


def dmd_edit_modes(model: DmdModel, threshold: float = 0.01, low=(1.0, 1.0, 1.0), high=(1.0, 1.0, 1.0),
                   dt: float = 1.0) -> torch.Tensor:
    """Edited modal buffer (Eq. edit_temporal) for dmd_predict(..., modal=...):
    per cluster (w, s_re, s_im) = (weight, scale of Re Omega, scale of Im Omega)."""
    out = torch.empty_like(model.modal)
    lo = (ctypes.c_double * 3)(*low)
    hi = (ctypes.c_double * 3)(*high)
    _check(lib().dmd_edit_modes(model.r, model.q, _ptr(model.modal), _ptr(out), float(threshold), lo, hi,
                                float(dt), _stream(model.modal.device)), "dmd_edit_modes")
    return out


def dmd_autotune_predict(model: DmdModel, ks, *, precision="mixed") -> tuple:
    """Tune the reconstruction kernel for this model's mode count on these
    frames; returns the chosen (chunk width, A stages, B ring entries)."""
    dev = model.Phi_R.device
    kt = _ks_tensor(ks, dev)
    K = kt.numel()
    out = torch.empty((K, round_up(model.n, 32)), dtype=torch.float32, device=dev)
    d = _pdesc(model, K, out.shape[1], precision, 0)
    ws = _pred_ws(d, dev)
    chosen = torch.zeros(3, dtype=torch.int32)
    _check(lib().dmd_autotune_predict(ctypes.byref(d), _ptr(model.Phi_R), _ptr(model.modal), _ptr(kt), _ptr(out),
                                      _ptr(ws), ws.numel(), _stream(dev), chosen.data_ptr()), "dmd_autotune_predict")
    return tuple(int(v) for v in chosen)


def dmd_predict_backward(model: DmdModel, ks, dOut: torch.Tensor, *, u: torch.Tensor | None = None,
                         precision="fp32", modal: torch.Tensor | None = None):
    """(d_modal, d_u) for dL/d(frames) = dOut (tensor (K, ldOut) float32)."""
    dev = model.Phi_R.device
    kt = _ks_tensor(ks, dev)
    _check_frames(model, kt.numel(), dOut, "dOut")
    _check_control(model, u)
    steps = 0 if u is None else u.shape[0]
    d = _pdesc(model, kt.numel(), dOut.shape[1], precision, steps)
    ws = _pred_ws(d, dev)
    md = _check_modal(model, modal)
    dmodal = torch.empty_like(md)
    du = None if u is None else torch.empty_like(u)
    _check(lib().dmd_predict_backward(ctypes.byref(d), _ptr(model.Phi_R), _ptr(md), _ptr(kt), _ptr(u), _ptr(dOut),
                                      _ptr(dmodal), _ptr(du), _ptr(ws), ws.numel(), _stream(dev)),
           "dmd_predict_backward")
    return dmodal, du


def dmd_predict_loss(model: DmdModel, ks, target: torch.Tensor, w: torch.Tensor, *, want_grad: bool = False,
                     u: torch.Tensor | None = None, precision="fp32", chunk: int = 50,
                     modal: torch.Tensor | None = None, loss: str = "quadratic", delta: float = 0.0):
    """Streamed L = sum_j w_j sum_i rho(x_{k_j,i} - target_i) (and its gradient):
    rho(e) = e^2 / 2 (loss="quadratic") or the Huber function of width delta
    (loss="huber")."""
    dev = model.Phi_R.device
    kt = _ks_tensor(ks, dev)
    _need_cuda(target, "target", torch.float32)
    _need_cuda(w, "w", torch.float64)
    if target.numel() < model.n or w.numel() < kt.numel():
        raise ValueError(f"target must hold n = {model.n} values and w K = {kt.numel()} weights")
    _check_control(model, u)
    steps = 0 if u is None else u.shape[0]
    d = _pdesc(model, kt.numel(), round_up(model.n, 32), precision, steps, chunk)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_predict_loss_workspace_bytes(ctypes.byref(d), 1 if want_grad else 0, ctypes.byref(nb)),
           "dmd_predict_loss_workspace_bytes")
    ws = _workspace(nb.value, dev)
    md = _check_modal(model, modal)
    dmodal = torch.empty_like(md) if want_grad else None
    du = torch.empty_like(u) if (want_grad and u is not None) else None
    opts = LossOpts(kind=LOSS_KINDS[loss], reserved=0, delta=float(delta))
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    _check(lib().dmd_predict_loss(ctypes.byref(d), _ptr(model.Phi_R), _ptr(md), _ptr(kt), _ptr(u), _ptr(target),
                                  _ptr(w), ctypes.byref(opts), 1 if want_grad else 0, _ptr(out), _ptr(dmodal),
                                  _ptr(du), _ptr(ws), ws.numel(), _stream(dev)), "dmd_predict_loss")
    return out, dmodal, du


def dmd_sketch_matrix(m: int, l: int, seed: int, device="cuda") -> torch.Tensor:
    """Philox Gaussian test matrix, tensor (l, m) float64 = column-major m x l."""
    out = torch.empty((l, m), dtype=torch.float64, device=device)
    _check(lib().dmd_sketch_matrix(m, l, seed, _ptr(out), _stream(out.device)), "dmd_sketch_matrix")
    return out


def dmd_philox_blocks(count: int, stream_id: int, key: int, device="cuda") -> torch.Tensor:
    out = torch.empty((count, 4), dtype=torch.int32, device=device)
    _check(lib().dmd_philox_blocks(count, stream_id, key, _ptr(out), _stream(out.device)), "dmd_philox_blocks")
    return out


def dmd_gemm_tall(A: torch.Tensor, n: int, B: torch.Tensor, *, precision="fp32", want_gram: bool = False,
                  out: torch.Tensor | None = None):
    """C = A B for tall A (tensor (Kd, lda) float32) and small B (tensor (N, Kd) float64)."""
    _need_cuda(A, "A", torch.float32)
    _need_cuda(B, "B", torch.float64)
    Kd, lda = A.shape
    N = B.shape[0]
    assert B.shape[1] == Kd
    dev = A.device
    ldc = round_up(n, 32)
    C = out if out is not None else torch.empty((N, ldc), dtype=torch.float32, device=dev)
    ldc = C.shape[1]
    gram = torch.empty((N, N), dtype=torch.float64, device=dev) if want_gram else None
    p = _prec(precision)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_gemm_tall_workspace_bytes(p, n, Kd, N, ctypes.byref(nb)), "dmd_gemm_tall_workspace_bytes")
    need = nb.value
    if want_gram:
        _check(lib().dmd_gemm_tn_workspace_bytes(p, n, N, N, ctypes.byref(nb)), "dmd_gemm_tn_workspace_bytes")
        need = max(need, nb.value)
    ws = _workspace(need, dev)
    _check(lib().dmd_gemm_tall(p, n, Kd, N, _ptr(A), lda, _ptr(B), _ptr(C), ldc, _ptr(gram), _ptr(ws),
                               ws.numel(), _stream(dev)), "dmd_gemm_tall")
    return (C, gram) if want_gram else C


def dmd_gemm_tn(A: torch.Tensor, B: torch.Tensor, n: int, *, precision="fp32") -> torch.Tensor:
    """C = A^T B over the tall dimension n; A (Ka, lda), B (N, ldb) float32; C (N, Ka) float64."""
    _need_cuda(A, "A", torch.float32)
    _need_cuda(B, "B", torch.float32)
    Ka, lda = A.shape
    N, ldb = B.shape
    dev = A.device
    p = _prec(precision)
    C = torch.empty((N, Ka), dtype=torch.float64, device=dev)
    nb = ctypes.c_size_t(0)
    _check(lib().dmd_gemm_tn_workspace_bytes(p, n, Ka, N, ctypes.byref(nb)), "dmd_gemm_tn_workspace_bytes")
    ws = _workspace(nb.value, dev)
    _check(lib().dmd_gemm_tn(p, n, Ka, N, _ptr(A), lda, _ptr(B), ldb, _ptr(C), _ptr(ws), ws.numel(), _stream(dev)),
           "dmd_gemm_tn")
    return C


class Batch:
    """Many scenes fitted and predicted in one call (dmd_fit_predict_batch).

    items: sequence of (S, n, r, seed, ks) with S a (m+1, ldS) float32 CUDA
    tensor of snapshots and ks the frame indices (or None for fit only).
    Outputs (models, frames) are allocated once; `run()` (re)executes the
    batch on the current stream and may be captured in a CUDA graph after the
    first call."""

    def __init__(self, items, *, lanes: int = 16, precision="fp32", oversample: int = 10, power_iters: int = 2):
        self.lanes = lanes
        self.models, self.frames, self._keep = [], [], []
        arr = (Scene * len(items))()
        for i, (S, n, r, seed, ks) in enumerate(items):
            _need_cuda(S, "S", torch.float32)
            dev = S.device
            m = S.shape[0] - 1
            ldPhi = round_up(n, 32)
            model = DmdModel(torch.empty((r, ldPhi), dtype=torch.float32, device=dev),
                             torch.empty(r * 4, dtype=torch.float64, device=dev),
                             torch.empty(INFO_WORDS, dtype=torch.int32, device=dev), n, r, 0)
            kt = None if ks is None else _ks_tensor(ks, dev)
            K = 0 if kt is None else kt.numel()
            out = torch.empty((K, ldPhi), dtype=torch.float32, device=dev) if K else None
            arr[i].fit = FitDesc(n=n, ldS=S.shape[1], ldPhi=ldPhi, m=m, r=r, oversample=min(oversample, m - r),
                                 power_iters=power_iters, q=0, precision=_prec(precision), seed=seed)
            arr[i].S, arr[i].Phi_R, arr[i].modal, arr[i].info = (_ptr(S), _ptr(model.Phi_R), _ptr(model.modal),
                                                                 _ptr(model.info))
            arr[i].K, arr[i].k, arr[i].out, arr[i].ldOut = K, _ptr(kt), _ptr(out), ldPhi
            self.models.append(model)
            self.frames.append(out)
            self._keep += [S, kt]
        self._arr = arr
        nb = ctypes.c_size_t(0)
        _check(lib().dmd_batch_workspace_bytes(len(items), arr, lanes, ctypes.byref(nb)), "dmd_batch_workspace_bytes")
        self._ws = _workspace(nb.value, items[0][0].device if items else torch.device("cuda"))

    def run(self):
        dev = self._ws.device
        _check(lib().dmd_fit_predict_batch(len(self.models), self._arr, self.lanes, _ptr(self._ws), self._ws.numel(),
                                           _stream(dev)), "dmd_fit_predict_batch")
        return self.models, self.frames


# ----------------------------------------------------------------- autograd


def _tie_pairs(dmodal: torch.Tensor, lam_im: torch.Tensor, r: int) -> torch.Tensor:
    """The kernels read a pair's eigenvalue from its first column only, so the
    gradient w.r.t. the second column's (Re, Im) entries is zero."""
    second = lam_im < 0
    g = dmodal.clone()
    g[:r][second] = 0
    g[r:2 * r][second] = 0
    g[3 * r:4 * r] = 0
    return g


class DmdPredict(torch.autograd.Function):
    """frames = dmd_predict(modal, u); differentiable in modal (lambda, beta, G) and u."""

    @staticmethod
    def forward(ctx, modal, u, model: DmdModel, ks, precision):
        kt = _ks_tensor(ks, modal.device)
        out = dmd_predict(model, kt, u=u, precision=precision, modal=modal.detach().contiguous())
        ctx.save_for_backward(modal.detach(), None if u is None else u.detach())
        ctx.model, ctx.kt, ctx.precision = model, kt, precision
        return out

    @staticmethod
    def backward(ctx, g):
        modal, u = ctx.saved_tensors
        dmodal, du = dmd_predict_backward(ctx.model, ctx.kt, g.contiguous(), u=u, precision=ctx.precision,
                                          modal=modal)
        r = ctx.model.r
        return _tie_pairs(dmodal, modal[r:2 * r], r), du, None, None, None


class DmdPredictLoss(torch.autograd.Function):
    """Streamed per-frame loss (frames recomputed in chunks, never stored)."""

    @staticmethod
    def forward(ctx, modal, u, model: DmdModel, ks, target, w, precision, chunk):
        kt = _ks_tensor(ks, modal.device)
        loss, dmodal, du = dmd_predict_loss(model, kt, target, w, want_grad=True, u=u, precision=precision,
                                            chunk=chunk, modal=modal.detach().contiguous())
        ctx.save_for_backward(dmodal, du if du is not None else torch.empty(0, device=modal.device),
                              modal[model.r:2 * model.r].detach())
        ctx.r, ctx.has_u = model.r, u is not None
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        dmodal, du, lam_im = ctx.saved_tensors
        gm = _tie_pairs(dmodal, lam_im, ctx.r) * g
        gu = (du * g) if ctx.has_u else None
        return gm, gu, None, None, None, None, None, None
