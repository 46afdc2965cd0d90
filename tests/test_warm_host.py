"""Host-side helpers of the warm-start evaluation (no GPU)."""
import numpy as np
import torch

import oracle as O
from paper_2003_07504_gb300 import synth, warmstart as ws


def test_stationarity_residual_is_half_the_energy_gradient():
    # the reported residual of the converged reference is max |dE/du| / 2 (Eq. 1): central
    # differences of the oracle's energy on a small image
    f = synth.preset_image(6, 7, 1, "small", 3)[0].astype(np.float64)
    u = f + 0.05 * synth.random_field(f.shape, seed=4).astype(np.float64)
    lam, p, eps = 1.3, 0.8, 1e-4
    h = 1e-6
    g = np.zeros_like(u)
    for i in range(u.shape[0]):
        for j in range(u.shape[1]):
            a, b = u.copy(), u.copy()
            a[i, j] += h
            b[i, j] -= h
            g[i, j] = (O.energy(a, f, lam, p, eps) - O.energy(b, f, lam, p, eps)) / (2 * h)
    r = ws.stationarity_residual(torch.from_numpy(u), torch.from_numpy(f), lam, p, eps)
    assert abs(r - 0.5 * np.abs(g).max()) <= 1e-5 * max(1.0, r)


def test_stationarity_residual_vanishes_at_a_fixed_point():
    f = np.full((1, 8, 8), 0.3)
    assert ws.stationarity_residual(torch.from_numpy(f), torch.from_numpy(f), 1.0, 0.8, 1e-4) == 0.0
