"""Small cases of the hot path's kernels, for profilers.

    python -m paper_2502_05339_gb300.profile_cases <case> [--rows N]

Each case builds seeded random operands of the 128^3 x 3 workload's column
counts on `cuda:0` with a reduced row count (default 1,048,576 rows: every
operand still exceeds the 129 MB L2, the whole case holds a few GB) and calls
the same entry point twice, so a profiler can skip the first (warm-up) launch:

  gram    snapshot Gram W = S^T S on the CUDA cores (201 columns, symmetric)
  tn      tensor-core reduction Q^T S (160 x 201 columns, BF16x3)
  gramq   tensor-core Gram Q^T Q (160 columns, BF16x3)
  sketch  tensor-core tall product X M (200 -> 160 columns, BF16x3)
  recon   reconstruction Phi_R C of 1000 frames (150 modes, BF16x3)
  advect  density advection (Sec. 7.2) on a 128^3 grid: a random 150-mode
          velocity model (RMS ~0.5 cells per unit step), 64 steps, frames rebuilt
          in batches of 64 (rows fixed by the grid; --rows is ignored)
  optdmd  OptDMD fit (Sec. 4.2) of a 3D 70^3 x 3 linear-modes scene (1,029,000
          rows; 200 snapshots, 75 pairs with stratified frequencies, rank 150,
          BF16x3 tall passes): the small FP64 loop is independent of the rows
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from paper_2502_05339_gb300 import dmd

M_SNAP, L_SKETCH, R_MODES, FRAMES = 200, 160, 150, 1000


def _rand(rows, cols, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randn((cols, rows), device="cuda", generator=g)


def _model(rows):
    P = _rand(rows, R_MODES, 3)
    rng = np.random.default_rng(4)
    lam = np.exp(rng.uniform(-0.02, 0, R_MODES // 2) + 1j * rng.uniform(0, np.pi, R_MODES // 2))
    modal = np.zeros(4 * R_MODES)
    modal[0:R_MODES:2], modal[1:R_MODES:2] = lam.real, lam.real
    modal[R_MODES:2 * R_MODES:2], modal[R_MODES + 1:2 * R_MODES:2] = lam.imag, -lam.imag
    modal[2 * R_MODES:3 * R_MODES] = rng.standard_normal(R_MODES)
    return dmd.DmdModel(P, torch.as_tensor(modal).cuda(), torch.zeros(8, dtype=torch.int32, device="cuda"),
                        rows, R_MODES, 0)


def run(case: str, rows: int, reps: int = 2):
    dmd.lib()
    if case == "gram":
        S = _rand(rows, M_SNAP + 1, 1)
        for _ in range(reps):
            dmd.dmd_gemm_tn(S, S, rows, precision="fp32")
    elif case in ("tn", "gramq"):
        Q = _rand(rows, L_SKETCH, 2)
        S = Q if case == "gramq" else _rand(rows, M_SNAP + 1, 1)
        for _ in range(reps):
            dmd.dmd_gemm_tn(Q, S, rows, precision="mixed")
    elif case == "sketch":
        X = _rand(rows, M_SNAP, 1)
        M = torch.randn((L_SKETCH, M_SNAP), dtype=torch.float64, device="cuda")
        for _ in range(reps):
            dmd.dmd_gemm_tall(X, rows, M, precision="mixed")
    elif case == "recon":
        model = _model(rows)
        ks = torch.arange(FRAMES, dtype=torch.int32, device="cuda")
        out = torch.empty((FRAMES, model.ldPhi), dtype=torch.float32, device="cuda")
        for _ in range(reps):
            dmd.dmd_predict(model, ks, precision="mixed", out=out)
    elif case == "advect":
        N = 128
        model = _model(3 * N ** 3)
        model.Phi_R.mul_(0.05)
        rho0 = torch.rand(N ** 3, device="cuda")
        for _ in range(reps):
            dmd.dmd_advect_density(model, rho0, N, 3, 64, 0.5, precision="mixed", chunk=64)
    elif case == "optdmd":
        import math
        from paper_2502_05339_gb300 import synth
        sc = synth.linear_modes_scene(70, 3, R_MODES // 2, M_SNAP, 1001, sigma_lo=-0.02, omega_hi=math.pi,
                                      stratified=True, noise=1e-4, nonlinear=1e-3, device="cuda")
        for _ in range(reps):
            dmd.dmd_fit_optdmd(sc.S, sc.n, R_MODES, precision="mixed", seed=1001).check()
    else:
        raise SystemExit(f"unknown case {case!r}")
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["gram", "tn", "gramq", "sketch", "recon", "optdmd", "advect"])
    ap.add_argument("--rows", type=int, default=1 << 20)
    args = ap.parse_args()
    run(args.case, args.rows)
    print("ok", args.case, args.rows)


if __name__ == "__main__":
    main()
