"""Shared helpers of the GPU parity tests (comparison metrics only)."""
import numpy as np
import torch

from oracle import dmd_oracle as O


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cols(t: torch.Tensor, n: int) -> np.ndarray:
    """(cols, ld) column-major tensor -> (n, cols) FP64 numpy matrix."""
    return t[:, :n].double().cpu().numpy().T


def match(lam_g, lam_o):
    """Greedy minimum-distance matching; returns the permutation p with
    lam_g[p[j]] ~ lam_o[j] and the max relative distance."""
    avail = list(range(len(lam_g)))
    perm = []
    worst = 0.0
    for v in lam_o:
        j = min(avail, key=lambda i: abs(lam_g[i] - v))
        worst = max(worst, abs(lam_g[j] - v) / max(abs(v), 1e-300))
        perm.append(j)
        avail.remove(j)
    return np.array(perm), worst


def eig_frob(lam_g, lam_o):
    """Relative Frobenius error of the eigenvalue vector after matching."""
    perm, _ = match(lam_g, lam_o)
    return rel(np.asarray(lam_g)[perm], lam_o)


def oracle_model(S64: np.ndarray, r: int):
    ref = O.exact_dmd(S64, r)
    PhiR, beta, kinds = O.to_real_form(ref["Phi"], ref["lam"], ref["b"])
    return ref, PhiR, beta, kinds


def gpu_kinds(lam: np.ndarray) -> np.ndarray:
    return O.pair_kinds(lam)


def mode_product_error(PhiR_g, beta_g, lam_g, PhiR_o, beta_o, lam_o):
    """Relative Frobenius error of the scale-free fields [phi_j b_j] over all
    modes (after eigenvalue matching), and the per-mode relative errors."""
    kg, ko = gpu_kinds(lam_g), gpu_kinds(lam_o)
    pg = O.mode_products(PhiR_g, beta_g, kg)
    po = O.mode_products(PhiR_o, beta_o, ko)
    hg = lam_g[kg != 2]
    ho = lam_o[ko != 2]
    perm, _ = match(hg, ho)
    errs = [rel(pg[:, perm[j]], po[:, j]) for j in range(po.shape[1])]
    frob = rel(pg[:, perm], po)
    return frob, np.array(errs)
