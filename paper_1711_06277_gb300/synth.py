"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds input generation only -- no step of the ray-tracing method. The
turbulent-cloud snapshots of Sec. 4.1 (Gaussian-random-field density with a k^-4 power
spectrum, many sources with a broad luminosity function) are not available, so these
generators stand in for them:

* ``lognormal_field``: a periodic Gaussian random field with P(k) ~ k^slope (k = 0
  removed), scaled to unit variance, exponentiated to a lognormal with log-standard
  deviation ``sigma_ln`` and renormalised to unit sample mean.
* ``power_law_luminosities``: dN/dL ~ L^-2 on [a, b] by inverse CDF, normalised to sum 1.
* ``uniform_positions`` / ``cell_centre_position``: source positions in a box.

Every generator takes an explicit seed and returns float64 numpy arrays; callers cast to
float32 where the library expects it. Grid arrays are shaped (nz, ny, nx) so that the
flat index is ``i + nx*(j + ny*k)`` (x fastest).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lognormal_field",
    "uniform_field",
    "power_law_luminosities",
    "uniform_positions",
    "cell_centre_position",
    "uniform_weights",
    "random_rotation",
    "bubble_neutral_fraction",
]


def lognormal_field(n: int, sigma_ln: float, seed: int, slope: float = -4.0) -> np.ndarray:
    """Lognormal density on an n^3 periodic grid, mean exactly 1, shape (n, n, n)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P(k)) with P ~ k^slope
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln**2)
    rho /= rho.mean()
    return rho


def uniform_field(n: int, value: float = 1.0) -> np.ndarray:
    return np.full((n, n, n), float(value))


def power_law_luminosities(count: int, seed: int, a: float = 1e-3, b: float = 1.0) -> np.ndarray:
    """dN/dL ~ L^-2 on [a, b] by inverse CDF, normalised so the luminosities sum to 1."""
    rng = np.random.default_rng(seed)
    u = rng.random(count)
    lum = 1.0 / (1.0 / a - u * (1.0 / a - 1.0 / b))
    return lum / lum.sum()


def uniform_positions(count: int, seed: int, lo=(0.0, 0.0, 0.0), side: float = 1.0,
                      margin: float = 1e-6) -> np.ndarray:
    """Uniform-random positions strictly inside the box [lo, lo + side]^3, shape (count, 3)."""
    rng = np.random.default_rng(seed)
    frac = margin + (1.0 - 2.0 * margin) * rng.random((count, 3))
    return np.asarray(lo, dtype=np.float64)[None, :] + side * frac


def cell_centre_position(n: int, seed: int, lo=(0.0, 0.0, 0.0), side: float = 1.0,
                         border: int = 0) -> np.ndarray:
    """Centre of a seeded random cell (cells at least ``border`` away from the faces)."""
    rng = np.random.default_rng(seed)
    ijk = rng.integers(border, n - border, size=3)
    dx = side / n
    return (np.asarray(lo, dtype=np.float64) + (ijk + 0.5) * dx)[None, :]


def uniform_weights(n: int, seed: int) -> np.ndarray:
    """Per-cell loss weights w ~ U[0, 1), shape (n, n, n)."""
    return np.random.default_rng(seed).random((n, n, n))


def force_weights(n: int, seed: int) -> np.ndarray:
    """Loss weights of the force, v ~ U[-1, 1) per component, shape (3, n, n, n) (float64)."""
    return np.random.default_rng(seed + 104729).uniform(-1.0, 1.0, size=(3, n, n, n))


def random_rotation(seed: int) -> np.ndarray:
    """A uniformly random proper rotation matrix (row-major 3x3), via QR of a Gaussian matrix."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def bubble_neutral_fraction(n: int, pos, L, r_max: float = 0.12, x_in: float = 1e-4,
                            x_out: float = 1.0, width: float = 1.5, side: float = 1.0) -> np.ndarray:
    """Neutral fraction with ionized bubbles around sources, shape (n, n, n), float64.

    A stand-in for the neutral fraction of a grid some time after its sources switched on
    (Sec. 3.3.1, 4): low (x_in) inside a sphere around each source, high (x_out) outside,
    with a transition ``width`` cells thick (logistic in the distance). Bubble radii grow
    like L^(1/3), r_max (box units) for the brightest source. Purely an input shape: no step
    of the ray-tracing method is used to make it."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(L, dtype=np.float64).reshape(-1)
    dx = side / n
    ion = np.zeros((n, n, n))  # ionized share in [0, 1], the largest over the bubbles
    radii = r_max * (L / L.max()) ** (1.0 / 3.0)
    c = (np.arange(n) + 0.5) * dx
    for p, r in zip(pos, radii):
        reach = r + 6.0 * width * dx
        lo = np.clip(np.floor((p - reach) / dx).astype(int), 0, n)
        hi = np.clip(np.ceil((p + reach) / dx).astype(int) + 1, 0, n)
        if np.any(hi <= lo):
            continue
        z, y, x = np.meshgrid(c[lo[2]:hi[2]], c[lo[1]:hi[1]], c[lo[0]:hi[0]], indexing="ij")
        d = np.sqrt((x - p[0]) ** 2 + (y - p[1]) ** 2 + (z - p[2]) ** 2)
        share = 1.0 / (1.0 + np.exp((d - r) / (width * dx)))
        sub = ion[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        np.maximum(sub, share, out=sub)
    return x_out - (x_out - x_in) * ion
