"""Seeded synthetic images standing in for the natural photographs the ILS paper
times and shows (it reports speed averaged over ten natural images per size).

This module only draws inputs.  It holds none of the smoothing arithmetic, and
both the CUDA path's tests and the CPU oracle's tests feed on it.

Image model: K Voronoi regions (nearest of K uniform sites, Euclidean) of
constant intensity U(0,1) drawn independently per channel; plus, per region, a
sinusoidal texture A*sin(2*pi*(x cos t + y sin t)/T + phase) with t ~ U(0,pi),
phase ~ U(0,2pi), T ~ U(Tmin,Tmax), shared by the channels; plus iid Gaussian
noise N(0, sigma^2) per pixel and channel; clipped to [0,1]; float32, planar
C x H x W.
"""
from __future__ import annotations

import numpy as np

# name: (K, A, Tmin, Tmax, sigma)
PRESETS = {
    "small": (12, 0.05, 4.0, 8.0, 0.02),      # 256 x 256 parity images
    "hd": (200, 0.05, 4.0, 8.0, 0.02),        # 1920 x 1080 headline images
    "uhd": (800, 0.05, 4.0, 16.0, 0.03),      # 3840 x 2160 sweep images
}


def _nearest_site(H: int, W: int, sy: np.ndarray, sx: np.ndarray) -> np.ndarray:
    """Label of the nearest site for every pixel centre (y, x)."""
    try:
        from scipy.spatial import cKDTree
        tree = cKDTree(np.stack([sy, sx], axis=1))
        yy, xx = np.mgrid[0:H, 0:W]
        _, lab = tree.query(np.stack([yy.ravel(), xx.ravel()], axis=1).astype(np.float64))
        return lab.reshape(H, W)
    except ImportError:  # pragma: no cover - scipy is present on every machine used here
        yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
        best = np.full((H, W), np.inf)
        lab = np.zeros((H, W), dtype=np.int64)
        for k in range(len(sy)):
            d = (yy - sy[k]) ** 2 + (xx - sx[k]) ** 2
            m = d < best
            best[m] = d[m]
            lab[m] = k
        return lab


def voronoi_texture(H: int, W: int, C: int = 1, *, K: int = 12, A: float = 0.05,
                    Tmin: float = 4.0, Tmax: float = 8.0, sigma: float = 0.02,
                    seed: int = 0) -> np.ndarray:
    """One C x H x W float32 image of the model above, fully determined by `seed`."""
    rng = np.random.default_rng(seed)
    sy = rng.uniform(0, H, K)
    sx = rng.uniform(0, W, K)
    val = rng.uniform(0, 1, (C, K))
    th = rng.uniform(0, np.pi, K)
    ph = rng.uniform(0, 2 * np.pi, K)
    T = rng.uniform(Tmin, Tmax, K)
    lab = _nearest_site(H, W, sy, sx)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    tex = A * np.sin(2 * np.pi * (xx * np.cos(th[lab]) + yy * np.sin(th[lab])) / T[lab] + ph[lab])
    img = val[:, lab] + tex[None]
    img += rng.normal(0.0, sigma, (C, H, W))
    return np.ascontiguousarray(np.clip(img, 0.0, 1.0), dtype=np.float32)


def preset_image(H: int, W: int, C: int, preset: str, seed: int) -> np.ndarray:
    K, A, Tmin, Tmax, sigma = PRESETS[preset]
    return voronoi_texture(H, W, C, K=K, A=A, Tmin=Tmin, Tmax=Tmax, sigma=sigma, seed=seed)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform float32 field (cotangents, directions, weights) from a seed."""
    return np.random.default_rng(seed).uniform(lo, hi, shape).astype(np.float32)
