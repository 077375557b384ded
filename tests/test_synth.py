"""The seeded input generators (no DMD arithmetic): the lean generator of
the large workload follows the same recipe as the full one, and the
pair-by-pair mode iterator gives the rows make_modes stacks."""
import math

import numpy as np
import torch

from paper_2502_05339_gb300 import synth


def test_mode_iterator_matches_make_modes():
    modes = synth.make_modes(12, 3, 3, 9)
    for j, (re, im) in enumerate(synth.iter_mode_pairs(12, 3, 3, 9)):
        assert torch.equal(modes[2 * j], re) and torch.equal(modes[2 * j + 1], im)


def test_lean_generator_matches_full_recipe():
    """Without noise (whose stream differs by construction) the lean
    generator's FP32 accumulation equals the FP64 recipe to FP32 rounding."""
    kw = dict(sigma_lo=-0.02, omega_hi=math.pi, stratified=True, nonlinear=1e-3)
    a = synth.linear_modes_scene(16, 3, 6, 40, 77, **kw)
    b = synth.linear_modes_scene_lean(16, 3, 6, 40, 77, batch_pairs=4, **kw)
    assert a.n == b.n and a.ld == b.ld
    np.testing.assert_allclose(a.lam_true, b.lam_true)
    d = (a.S[:, :a.n].double() - b.S[:, :b.n].double()).norm() / a.S[:, :a.n].double().norm()
    assert float(d) < 1e-6


def test_lean_generator_noise_level():
    kw = dict(sigma_lo=-0.02, omega_hi=math.pi, stratified=True)
    a = synth.linear_modes_scene_lean(12, 3, 4, 20, 5, **kw)
    b = synth.linear_modes_scene_lean(12, 3, 4, 20, 5, noise=1e-3, **kw)
    diff = (b.S[:, :b.n] - a.S[:, :a.n]).double()
    assert abs(float(diff.std()) - 1e-3) < 1e-4
    rms = float(a.S[:, :a.n].double().pow(2).mean().sqrt())
    assert abs(rms - 1.0) < 1e-6            # signal scaled to RMS 1 over the window
