"""Seeded input generators (numpy PCG64).

Everything here is input construction for the multi-image super-resolution workloads of
Sec. 4 of the paper (CT projections captured with a subpixel detector shift, Sec. 3.2 and
Fig. 4): an attenuation phantom standing in for the paper's cylinders and QRM bar targets,
the detector shift patterns, the Gaussian PSF taps, additive Gaussian noise and Poisson
detector counts.  The image-formation operator y_k = D B M_k x itself is NOT here; callers
apply it with the oracle (tests) or with the library's forward operator (benchmark).
"""
from __future__ import annotations

import numpy as np

# One fixed seed per workload.
CONFIG_SEEDS = {
    "tiny": 20210810,        # 4 x 64^2 -> 128^2
    "detector": 20210811,    # 4 x 2048^2 -> 4096^2
    "batch": 20210812,       # 64 uneven projections, f = 2 and 3
    "precision": 20210813,   # 4 x 3072^2 uint16 counts
    "serving": 20210814,     # streamed projections
}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def phantom(H: int, W: int, seed: int) -> np.ndarray:
    """HR attenuation line-integral image, float64, values in [0, 4].

    * 12-40 random spheres, each contributing the line integral of a homogeneous ball,
      peak * sqrt(1 - rho^2 / R^2), with peak ~ U(0.3, 1.5) and
      R ~ U(0.02, 0.12) * min(H, W)  (resolution-independent shapes);
    * 3-6 groups of 5 bars (value 1.0), bar period ~ U{2..16} HR px, half-period wide,
      horizontal or vertical, standing in for a QRM bar-pattern target;
    * summed and clipped to [0, 4].
    """
    rng = _rng(seed)
    x = np.zeros((H, W), dtype=np.float64)
    m = min(H, W)
    n_disks = int(rng.integers(12, 41))
    for _ in range(n_disks):
        cy = rng.uniform(0, H)
        cx = rng.uniform(0, W)
        rad = rng.uniform(0.02, 0.12) * m
        peak = rng.uniform(0.3, 1.5)
        y0, y1 = max(0, int(np.floor(cy - rad))), min(H, int(np.ceil(cy + rad)) + 1)
        x0, x1 = max(0, int(np.floor(cx - rad))), min(W, int(np.ceil(cx + rad)) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = (np.arange(y0, y1) + 0.5 - cy)[:, None]
        xx = (np.arange(x0, x1) + 0.5 - cx)[None, :]
        rho2 = (yy * yy + xx * xx) / (rad * rad)
        x[y0:y1, x0:x1] += peak * np.sqrt(np.clip(1.0 - rho2, 0.0, None))
    n_groups = int(rng.integers(3, 7))
    for _ in range(n_groups):
        period = int(rng.integers(2, 17))
        width = max(1, period // 2)
        length = max(2, int(rng.uniform(0.05, 0.25) * m))
        span = 5 * period
        vertical = bool(rng.random() < 0.5)
        if vertical:  # bars are vertical stripes: run along rows, repeat along columns
            oy = int(rng.integers(0, max(1, H - length)))
            ox = int(rng.integers(0, max(1, W - span)))
            for b in range(5):
                c0 = ox + b * period
                x[oy:oy + length, c0:c0 + width] += 1.0
        else:
            oy = int(rng.integers(0, max(1, H - span)))
            ox = int(rng.integers(0, max(1, W - length)))
            for b in range(5):
                r0 = oy + b * period
                x[r0:r0 + width, ox:ox + length] += 1.0
    return np.clip(x, 0.0, 4.0)


def gaussian_psf(size: int = 5, sigma: float = 0.5) -> np.ndarray:
    """size x size Gaussian PSF taps (sigma in HR px), float64, summing to 1."""
    if size % 2 != 1:
        raise ValueError("PSF size must be odd")
    r = size // 2
    a = np.arange(-r, r + 1, dtype=np.float64)
    if sigma <= 0:
        g = (a == 0).astype(np.float64)
    else:
        g = np.exp(-(a * a) / (2.0 * sigma * sigma))
    k = np.outer(g, g)
    return k / k.sum()


def phase_shifts(f: int) -> list[tuple[float, float]]:
    """All f*f subpixel detector positions (dx, dy) = (a/f, b/f) LR px, row-major in b."""
    return [(a / f, b / f) for b in range(f) for a in range(f)]


def half_pixel_shifts() -> list[tuple[float, float]]:
    """The 4 half-pixel detector positions (dx, dy) of Sec. 3.2: (0,0), (1/2,0), (0,1/2), (1/2,1/2)."""
    return [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]


def third_pixel_shifts() -> list[tuple[float, float]]:
    """The 9 third-pixel positions used for 3x magnification (Sec. 4.1.4)."""
    return phase_shifts(3)


def gaussian_noise(shape, sigma: float, seed: int) -> np.ndarray:
    return _rng(seed).normal(0.0, sigma, size=shape)


def poisson_counts(line_integrals: np.ndarray, flat_field: float, seed: int) -> np.ndarray:
    """Detector counts clamp(Poisson(I0 * exp(-m)), 1, 65535) as uint16 (Beer-Lambert)."""
    lam = flat_field * np.exp(-np.asarray(line_integrals, dtype=np.float64))
    c = _rng(seed).poisson(lam)
    return np.clip(c, 1, 65535).astype(np.uint16)


def impulse_noise(shape, frac: float, amp: float, seed: int) -> np.ndarray:
    """Sparse outliers (defective or saturated detector pixels): a fraction `frac` of the
    samples, chosen at random, offset by +-amp; zero elsewhere."""
    rng = _rng(seed)
    hit = rng.uniform(size=shape) < frac
    sign = np.where(rng.uniform(size=shape) < 0.5, -1.0, 1.0)
    return np.where(hit, amp * sign, 0.0)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return _rng(seed).uniform(lo, hi, size=shape)


def smooth_field(H: int, W: int, seed: int, n_waves: int = 6) -> np.ndarray:
    """Sum of a few random plane waves: a smooth, non-constant test image."""
    rng = _rng(seed)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    out = np.zeros((H, W))
    for _ in range(n_waves):
        ky, kx = rng.uniform(-0.2, 0.2, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        out += rng.uniform(0.1, 0.5) * np.cos(ky * yy + kx * xx + ph)
    return out


def batch_rois(seed: int, n: int = 64, lo: int = 512, hi: int = 2048):
    """Uneven projection batch: LR ROI sizes h, w ~ U{lo..hi}; first half f=2/K=4 with
    half-pixel shifts, second half f=3/K=9 with third-pixel shifts."""
    rng = _rng(seed)
    out = []
    for i in range(n):
        h = int(rng.integers(lo, hi + 1))
        w = int(rng.integers(lo, hi + 1))
        if i < n // 2:
            out.append({"h": h, "w": w, "f": 2, "shifts": half_pixel_shifts(), "seed": int(seed) * 1000 + i})
        else:
            out.append({"h": h, "w": w, "f": 3, "shifts": third_pixel_shifts(), "seed": int(seed) * 1000 + i})
    return out
