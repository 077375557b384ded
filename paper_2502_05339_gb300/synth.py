"""Seeded synthetic snapshot generators (inputs only; no DMD arithmetic).

This module is the one place that both the CUDA path's tests/benchmarks and the
FP64 oracle take their inputs from.  It builds velocity snapshots on a periodic
staggered (MAC) grid, the state layout of Sec. 4.1 of the paper: every snapshot
is the stacked vector of face velocities (Eq. "measurement vector", Sec. 3).

Recipe (the paper's scenes and solvers are not available, so these stand in):

* spatial modes are discrete curls of random low-wavenumber Fourier potentials
  (a nodal stream function in 2D, an edge vector potential in 3D), so every
  field is discretely divergence-free up to rounding (Sec. 4.5);
* Fourier coefficients are complex Gaussians scaled by 1/(1+|kappa|^2/kc^2) for
  integer wavevectors with |kappa|_inf <= kc (a band-limited, mildly decaying
  spectrum: the curl image has ~2(2kc+1)^3 dimensions in 3D, (2kc+1)^2 in 2D,
  so a few hundred random modes stay well conditioned);
* a complex mode is curl(psi_re) + i curl(psi_im), scaled to unit RMS;
* eigenvalues lambda_j = exp(sigma_j + i omega_j) in conjugate pairs, real
  amplitudes a_j ~ N(0, 1);
* snapshot x_k = sum_j 2 a_j |lambda_j|^k (Re phi_j cos(k w_j) - Im phi_j sin(k w_j)),
  optionally plus a weak quadratic term and Gaussian noise.

All small random draws (spectra, eigenvalues, amplitudes, blob centres) use
NumPy's PCG64 seeded by the caller, so they are identical on every machine.
Dense noise is drawn with torch's generator on the device the data is built
on (seed + 7), which is deterministic per device type.

Matrices are stored column-major the way the C ABI wants them: a torch tensor
of shape (cols, ld) whose row c is column c of the matrix, ld >= n padded to a
multiple of 32 floats.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

LD_ALIGN = 32  # floats: 128-byte column starts


def round_up(x: int, a: int) -> int:
    return (x + a - 1) // a * a


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# periodic MAC grid: discrete curl (fields) and divergence (checks)
# ----------------------------------------------------------------------------

def _fd(a: torch.Tensor, dim: int) -> torch.Tensor:
    """Forward difference with periodic wrap: a[i+1] - a[i]."""
    return torch.roll(a, -1, dims=dim) - a


def curl2d(psi: torch.Tensor) -> torch.Tensor:
    """Face velocities (u on x-faces, v on y-faces) of a nodal stream function.

    psi has shape (..., N, N); returns (..., 2*N*N) = [u.ravel(), v.ravel()].
    """
    u = _fd(psi, -1)          # d psi / dy
    v = -_fd(psi, -2)         # -d psi / dx
    return torch.cat([u.flatten(-2), v.flatten(-2)], dim=-1)


def div2d(x: torch.Tensor, N: int) -> torch.Tensor:
    """Cell-centred discrete divergence of stacked face velocities (..., 2N^2).

    u[i, j] sits on the face (i, j+1/2) and v[i, j] on (i+1/2, j), so the
    divergence of cell (i+1/2, j+1/2) takes forward differences of both.
    """
    u = x[..., : N * N].unflatten(-1, (N, N))
    v = x[..., N * N:].unflatten(-1, (N, N))
    return (_fd(u, -2) + _fd(v, -1)).flatten(-2)


def curl3d(ax: torch.Tensor, ay: torch.Tensor, az: torch.Tensor) -> torch.Tensor:
    """Face velocities of an edge vector potential on a periodic N^3 grid.

    Inputs have shape (..., N, N, N) indexed [x, y, z]; returns (..., 3N^3).
    """
    ux = _fd(az, -2) - _fd(ay, -1)
    uy = _fd(ax, -1) - _fd(az, -3)
    uz = _fd(ay, -3) - _fd(ax, -2)
    return torch.cat([ux.flatten(-3), uy.flatten(-3), uz.flatten(-3)], dim=-1)


def div3d(x: torch.Tensor, N: int) -> torch.Tensor:
    c = N ** 3
    ux = x[..., :c].unflatten(-1, (N, N, N))
    uy = x[..., c:2 * c].unflatten(-1, (N, N, N))
    uz = x[..., 2 * c:].unflatten(-1, (N, N, N))
    return (_fd(ux, -3) + _fd(uy, -2) + _fd(uz, -1)).flatten(-3)


# ----------------------------------------------------------------------------
# random potentials and modes
# ----------------------------------------------------------------------------

def _low_k_coefficients(g: np.random.Generator, dim: int, kc: int) -> tuple[np.ndarray, np.ndarray]:
    """Integer wavevectors |kappa|_inf <= kc and complex Gaussian coefficients."""
    ks = np.arange(-kc, kc + 1)
    grids = np.meshgrid(*([ks] * dim), indexing="ij")
    kap = np.stack([q.ravel() for q in grids], axis=1)
    amp = 1.0 / (1.0 + (kap.astype(np.float64) ** 2).sum(1) / float(kc * kc))
    c = (g.standard_normal(len(kap)) + 1j * g.standard_normal(len(kap))) * amp
    return kap, c


def fourier_potential(g: np.random.Generator, N: int, dim: int, kc: int,
                      device, dtype=torch.float64) -> torch.Tensor:
    """Real periodic field sum_kappa Re(c_kappa exp(2 pi i kappa.x / N))."""
    kap, c = _low_k_coefficients(g, dim, kc)
    spec = torch.zeros((N,) * dim, dtype=torch.complex128, device=device)
    idx = tuple(torch.as_tensor(kap[:, d] % N, device=device) for d in range(dim))
    spec.index_put_(idx, torch.as_tensor(c, device=device), accumulate=True)
    # ifftn includes 1/N^dim; undo it so the field's magnitude is O(1)
    f = torch.fft.ifftn(spec).real * float(N ** dim)
    return f.to(dtype)


def iter_mode_pairs(N: int, dim: int, npairs: int, seed: int, kc: int | None = None,
                    device="cpu", dtype=torch.float64):
    """Yields (Re phi_j, Im phi_j) of each complex divergence-free mode in
    turn (unit RMS per complex mode): the rows make_modes stacks, one pair
    at a time for grids where all of them do not fit at once."""
    if kc is None:
        kc = 8 if dim == 2 else 4
    g = rng(seed)
    for _ in range(npairs):
        parts = []
        for _ in range(2):  # real and imaginary potentials
            if dim == 2:
                parts.append(curl2d(fourier_potential(g, N, 2, kc, device)))
            else:
                a = [fourier_potential(g, N, 3, kc, device) for _ in range(3)]
                parts.append(curl3d(*a))
        re, im = parts
        rms = torch.sqrt((re * re + im * im).mean())
        yield (re / rms).to(dtype), (im / rms).to(dtype)


def make_modes(N: int, dim: int, npairs: int, seed: int, kc: int | None = None,
               device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Complex divergence-free modes as a real (2*npairs, n) tensor.

    Row 2j is Re(phi_j), row 2j+1 is Im(phi_j); each complex mode has unit RMS.
    """
    n = dim * N ** dim
    out = torch.empty((2 * npairs, n), dtype=dtype, device=device)
    for j, (re, im) in enumerate(iter_mode_pairs(N, dim, npairs, seed, kc, device, dtype)):
        out[2 * j] = re
        out[2 * j + 1] = im
    return out


def draw_spectrum(g: np.random.Generator, npairs: int, sigma_lo: float, omega_hi: float,
                  stratified: bool = False):
    """sigma ~ U(sigma_lo, 0), a ~ N(0, 1) and omega in (0, omega_hi):
    uniform, or stratified -- one uniform draw inside each of npairs equal
    cells -- so that no two pairs share a frequency resolution cell."""
    sigma = g.uniform(sigma_lo, 0.0, npairs)
    if stratified:
        omega = (np.arange(npairs) + g.uniform(0.0, 1.0, npairs)) * (omega_hi / npairs)
        omega = omega[g.permutation(npairs)]
    else:
        omega = g.uniform(0.0, omega_hi, npairs)
    a = g.standard_normal(npairs)
    return sigma, omega, a


def time_factors(sigma, omega, a, ks) -> np.ndarray:
    """(2P, K) real factors T with x_k = Phi_true_rows^T T[:, k] (FP64, host)."""
    ks = np.asarray(ks, dtype=np.float64)
    mag = np.exp(np.outer(sigma, ks))
    T = np.empty((2 * len(sigma), len(ks)))
    T[0::2] = 2.0 * a[:, None] * mag * np.cos(np.outer(omega, ks))
    T[1::2] = -2.0 * a[:, None] * mag * np.sin(np.outer(omega, ks))
    return T


def prolong(S: torch.Tensor, N: int, dim: int, factor: int) -> torch.Tensor:
    """Piecewise-constant prolongation of every snapshot (rows of S, (count, ld)
    float32, dim stacked components of an N^dim grid) to the (factor N)^dim
    grid: the stand-in for a low-resolution simulation's fields given on the
    high-resolution grid (the upsampling inputs L_t).  Returns (count, ld')
    float32 with ld' = round_up(dim (factor N)^dim, 32), zero padded."""
    count = S.shape[0]
    n = dim * N ** dim
    Nf = factor * N
    nf = dim * Nf ** dim
    out = torch.zeros((count, round_up(nf, 32)), dtype=torch.float32, device=S.device)
    comp = S[:, :n].reshape((count, dim) + (N,) * dim)
    for ax in range(dim):
        comp = comp.repeat_interleave(factor, dim=2 + ax)
    out[:, :nf] = comp.reshape(count, nf)
    return out


# ----------------------------------------------------------------------------
# scene containers
# ----------------------------------------------------------------------------

@dataclass
class Scene:
    """One synthetic snapshot sequence S = [x_0 .. x_m] and its ground truth."""
    name: str
    N: int
    dim: int
    n: int
    m: int
    ld: int
    S: torch.Tensor                 # (m+1, ld) float32, column-major n x (m+1)
    lam_true: np.ndarray            # (2P,) complex, conjugate pairs adjacent
    modes_true: torch.Tensor | None = None  # (2P, n) real rows [Re, Im] (FP64)
    amps_true: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    def X(self, dtype=torch.float64) -> torch.Tensor:
        """(n, m+1) dense copy of the snapshot matrix (host, for the oracle)."""
        return self.S[:, : self.n].to("cpu", dtype).T.contiguous()


def _pack(cols: torch.Tensor, ld: int) -> torch.Tensor:
    """(ncols, n) rows -> (ncols, ld) float32 zero-padded column-major storage."""
    out = torch.zeros((cols.shape[0], ld), dtype=torch.float32, device=cols.device)
    out[:, : cols.shape[1]] = cols.to(torch.float32)
    return out


def linear_modes_scene(N: int, dim: int, npairs: int, m: int, seed: int, *,
                       sigma_lo: float = -0.05, omega_hi: float = math.pi / 4,
                       noise: float = 0.0, nonlinear: float = 0.0, stratified: bool = False,
                       device="cpu", name: str = "", keep_fp64: bool = False) -> Scene:
    """Sum of `npairs` conjugate-pair divergence-free modes (configs 0, 1, 4).

    The noise-free signal is scaled to RMS 1 over the window; then the optional
    quadratic term (products of 4 pairs, relative scale `nonlinear`) and
    Gaussian noise of absolute std `noise` are added.  With keep_fp64 the
    unrounded FP64 snapshot matrix (n x (m+1)) is kept in extra["S64"].
    """
    g = rng(seed)
    n = dim * N ** dim
    ld = round_up(n, LD_ALIGN)
    modes = make_modes(N, dim, npairs, seed + 1, device=device)
    sigma, omega, a = draw_spectrum(g, npairs, sigma_lo, omega_hi, stratified)
    ks = np.arange(m + 1)
    T = torch.as_tensor(time_factors(sigma, omega, a, ks), device=device)
    sig = T.T @ modes                                   # (m+1, n) FP64
    scale = 1.0 / float(torch.sqrt((sig * sig).mean()))
    sig *= scale
    if nonlinear > 0.0:
        sel = g.choice(npairs, size=min(4, npairs), replace=False)
        rows = torch.as_tensor(np.stack([2 * sel, 2 * sel + 1], 1).ravel(), device=device)
        Tsel = T[rows]                                   # (2*4, m+1)
        msel = modes[rows]                               # (2*4, n)
        quad = torch.empty_like(sig)
        for k in range(m + 1):
            f = (Tsel[0::2, k, None] * msel[0::2] + Tsel[1::2, k, None] * msel[1::2]) * scale
            acc = torch.zeros(n, dtype=sig.dtype, device=device)
            for i in range(len(sel)):
                for j in range(i, len(sel)):
                    acc += f[i] * f[j]
            quad[k] = acc
        quad *= nonlinear / float(torch.sqrt((quad * quad).mean()))
        sig += quad
    if noise > 0.0:
        tg = torch.Generator(device=device)
        tg.manual_seed(seed + 7)
        sig += noise * torch.randn(sig.shape, generator=tg, dtype=torch.float32,
                                   device=device).to(sig.dtype)
    lam = np.exp(sigma + 1j * omega)
    lam_pairs = np.empty(2 * npairs, dtype=complex)
    lam_pairs[0::2], lam_pairs[1::2] = lam, lam.conj()
    extra = dict(sigma=sigma, omega=omega, scale=scale, noise=noise, nonlinear=nonlinear)
    if keep_fp64:
        extra["S64"] = sig.T.to("cpu").numpy().copy()
    return Scene(name or f"linear{dim}d_{N}", N, dim, n, m, ld, _pack(sig, ld),
                 lam_pairs, modes, a * scale, extra=extra)


def linear_modes_scene_lean(N: int, dim: int, npairs: int, m: int, seed: int, *,
                            sigma_lo: float = -0.05, omega_hi: float = math.pi / 4,
                            noise: float = 0.0, nonlinear: float = 0.0, stratified: bool = False,
                            device="cpu", name: str = "", batch_pairs: int = 10) -> Scene:
    """The recipe of linear_modes_scene for grids whose FP64 intermediates do
    not fit in memory: the snapshots are accumulated in FP32 on `device` from
    batches of `batch_pairs` modes (one FP32 matrix product per batch), then
    scaled to RMS 1; the quadratic term (same selection of 4 pairs, relative
    scale `nonlinear`) and the noise are added row by row.  The modes are not
    kept (modes_true is None)."""
    g = rng(seed)
    n = dim * N ** dim
    ld = round_up(n, LD_ALIGN)
    sigma, omega, a = draw_spectrum(g, npairs, sigma_lo, omega_hi, stratified)
    sel = list(g.choice(npairs, size=min(4, npairs), replace=False)) if nonlinear > 0.0 else []
    ks = np.arange(m + 1)
    T = torch.as_tensor(time_factors(sigma, omega, a, ks), device=device)        # (2P, m+1) FP64
    S = torch.zeros((m + 1, ld), dtype=torch.float32, device=device)
    kept = {}
    rows, fields = [], []
    for j, (re, im) in enumerate(iter_mode_pairs(N, dim, npairs, seed + 1, device=device)):
        if j in sel:
            kept[j] = (re, im)
        rows += [2 * j, 2 * j + 1]
        fields += [re.to(torch.float32), im.to(torch.float32)]
        if len(fields) == 2 * batch_pairs or j == npairs - 1:
            M = torch.stack(fields)                                             # (2b, n) FP32
            Tb = T[rows].to(torch.float32)                                      # (2b, m+1)
            S[:, :n].addmm_(Tb.T, M)
            rows, fields = [], []
            del M
    ss = sum(float((S[k, :n].double() ** 2).sum()) for k in range(m + 1))
    scale = 1.0 / math.sqrt(ss / ((m + 1) * n))
    S[:, :n] *= scale
    if sel:
        def quad_row(k):
            f = [(T[2 * j, k] * kept[j][0] + T[2 * j + 1, k] * kept[j][1]) * scale for j in sel]
            acc = torch.zeros(n, dtype=torch.float64, device=device)
            for i in range(len(f)):
                for jj in range(i, len(f)):
                    acc += f[i] * f[jj]
            return acc
        qq = sum(float((quad_row(k) ** 2).sum()) for k in range(m + 1))
        qs = nonlinear / math.sqrt(qq / ((m + 1) * n))
        for k in range(m + 1):
            S[k, :n] += (qs * quad_row(k)).to(torch.float32)
    if noise > 0.0:
        tg = torch.Generator(device=device)
        tg.manual_seed(seed + 7)
        for k in range(m + 1):
            S[k, :n] += noise * torch.randn(n, generator=tg, dtype=torch.float32, device=device)
    lam = np.exp(sigma + 1j * omega)
    lam_pairs = np.empty(2 * npairs, dtype=complex)
    lam_pairs[0::2], lam_pairs[1::2] = lam, lam.conj()
    extra = dict(sigma=sigma, omega=omega, scale=scale, noise=noise, nonlinear=nonlinear)
    return Scene(name or f"linear{dim}d_{N}_lean", N, dim, n, m, ld, S, lam_pairs, None, a * scale, extra=extra)


# ----------------------------------------------------------------------------
# the benchmark configurations (sizes from the workload definitions)
# ----------------------------------------------------------------------------

def config0(seed: int = 1000, device="cpu", noise: float = 1e-8, keep_fp64: bool = False) -> Scene:
    """2D 64x64 grid x 2 components (n = 8192), m = 100, 20 modes, noise 1e-8."""
    return linear_modes_scene(64, 2, 10, 100, seed, noise=noise, device=device,
                              name="cfg0_2d64", keep_fp64=keep_fp64)


def config1(seed: int = 1001, device="cpu", N: int = 128, m: int = 200, literal: bool = False) -> Scene:
    """3D 128^3 x 3 (n = 6,291,456), m = 200, 150 modes, sigma ~ U(-0.02, 0),
    quadratic term 1e-3, noise 1e-4.

    With 75 pairs and 200 snapshots the frequencies must fill the half circle
    to be resolvable (a window of m samples separates about m / (2 pi) per
    radian), so by default omega is stratified over (0, pi).  literal=True
    draws omega ~ U(0, pi/4) as for config 0; that data has numerical rank
    of about 60, so a rank-150 fit of it regresses noise."""
    if literal:
        return linear_modes_scene(N, 3, 75, m, seed, sigma_lo=-0.02, noise=1e-4, nonlinear=1e-3,
                                  device=device, name=f"cfg1lit_3d{N}")
    return linear_modes_scene(N, 3, 75, m, seed, sigma_lo=-0.02, omega_hi=math.pi, stratified=True,
                              noise=1e-4, nonlinear=1e-3, device=device, name=f"cfg1_3d{N}")


def blob_forces(N: int, dim: int, q: int, g: np.random.Generator, width: float = 6.0,
                device="cpu") -> torch.Tensor:
    """q smooth force fields: unit random direction x periodic Gaussian blob."""
    n = dim * N ** dim
    out = torch.empty((q, n), dtype=torch.float64, device=device)
    ax = torch.arange(N, dtype=torch.float64, device=device)
    for c in range(q):
        centre = g.uniform(0, N, dim)
        direction = g.standard_normal(dim)
        direction /= np.linalg.norm(direction)
        d2 = torch.zeros((N,) * dim, dtype=torch.float64, device=device)
        for d in range(dim):
            dd = torch.remainder(ax - centre[d] + N / 2, N) - N / 2
            shape = [1] * dim
            shape[d] = N
            d2 = d2 + (dd * dd).reshape(shape)
        blob = torch.exp(-d2 / (2 * width * width))
        out[c] = torch.cat([direction[d] * blob.flatten() for d in range(dim)])
    return out


def piecewise_controls(g: np.random.Generator, q: int, steps: int, hold: int = 20) -> np.ndarray:
    """(q, steps) amplitudes ~ U(-1, 1), held constant for `hold` steps."""
    nblk = (steps + hold - 1) // hold
    blk = g.uniform(-1.0, 1.0, (q, nblk))
    return np.repeat(blk, hold, axis=1)[:, :steps]


def controlled_scene(N: int, dim: int, npairs: int, m: int, q: int, seed: int,
                     device="cpu", sigma_lo: float = -0.02, stratified: bool = True) -> Scene:
    """DMDc data (config 2 recipe): latent z_{k+1} = L z_k + P F u_k, x_k = Phi z_k.

    Phi are `npairs` conjugate-pair curl modes in real 2x2 form, F are q blob
    force fields, P F is the least-squares projection of F onto span(Phi), so
    every snapshot stays in span(Phi) and divergence-free.  No noise.
    """
    g = rng(seed)
    n = dim * N ** dim
    ld = round_up(n, LD_ALIGN)
    modes = make_modes(N, dim, npairs, seed + 1, device=device)     # (2P, n)
    sigma, omega, a = draw_spectrum(g, npairs, sigma_lo, math.pi / 4, stratified)
    F = blob_forces(N, dim, q, g, device=device)                     # (q, n)
    gram = modes @ modes.T
    PF = torch.linalg.solve(gram, modes @ F.T)                       # (2P, q)
    U = piecewise_controls(g, q, m)                                  # (q, m)
    lam = np.exp(sigma + 1j * omega)
    # real 2x2 blocks on (c0, c1) = (2 Re z, -2 Im z), x = sum_j Re(phi_j) c0 + Im(phi_j) c1
    L = np.zeros((2 * npairs, 2 * npairs))
    for j in range(npairs):
        lr, li = lam[j].real, lam[j].imag
        L[2 * j:2 * j + 2, 2 * j:2 * j + 2] = [[lr, li], [-li, lr]]
    z = np.zeros((2 * npairs, m + 1))
    z[:, 0] = np.repeat(a, 2) * np.tile([1.0, 0.0], npairs)
    PFh = PF.cpu().numpy()
    for k in range(m):
        z[:, k + 1] = L @ z[:, k] + PFh @ U[:, k]
    sig = torch.as_tensor(z.T, device=device) @ modes                # (m+1, n)
    S64 = sig.T.to("cpu").numpy().copy() if n * (m + 1) <= 50_000_000 else None
    lam_pairs = np.empty(2 * npairs, dtype=complex)
    lam_pairs[0::2], lam_pairs[1::2] = lam, lam.conj()
    return Scene(f"dmdc{dim}d_{N}", N, dim, n, m, ld, _pack(sig, ld), lam_pairs, modes, a,
                 extra=dict(U=U, F=F, PF=PFh, L=L, z=z, S64=S64))


def config2(seed: int = 1002, device="cpu", N: int = 96, m: int = 300) -> Scene:
    """DMDc on 96^3 x 3 (n = 2,654,208), m = 300, q = 8 blob forces, 100 modes."""
    return controlled_scene(N, 3, 50, m, 8, seed, device=device)


def random_sketch(m: int, l: int, seed: int) -> np.ndarray:
    """Gaussian N(0,1) test matrix (m x l), drawn on the host with PCG64."""
    return rng(seed).standard_normal((m, l))


def config4(seed: int = 1004, device="cpu", N: int = 256, m: int = 300) -> Scene:
    """3D 256^3 x 3 (n = 50,331,648), m = 300 (~60 GB of FP32 snapshots), data
    as config 1: 75 pairs, sigma ~ U(-0.02, 0), frequencies stratified over
    (0, pi), quadratic term 1e-3, noise 1e-4; built by the lean generator."""
    return linear_modes_scene_lean(N, 3, 75, m, seed, sigma_lo=-0.02, omega_hi=math.pi, stratified=True,
                                   noise=1e-4, nonlinear=1e-3, device=device, name=f"cfg4_3d{N}")
