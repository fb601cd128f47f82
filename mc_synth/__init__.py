"""Seeded synthetic inputs for motion-compensated CT reconstruction.

This module is the ONLY code shared between the FP64 oracle (``oracle/``),
the CUDA path (``paper_2410_10503_gb300``), the tests and ``bench.py``.
It draws random inputs and nothing else: it holds none of the method's
arithmetic (no ray transform, no warp, no proximal step, no sampling of
gates).  Random numbers that the method itself consumes (the measurement
noise of the gated data model, Sec. II-A) are drawn here and passed in as
inputs; the gate draw of Algorithm 1 step (ii) uses a counter-based
generator that each side implements on its own.

The paper's own data (a walnut slice and a chest slice, Sec. III) are not
available; the workloads below stand in for them with the sizes and the
kind of motion the paper describes (rigid rotation + translation, and a
smooth non-rigid field), on random-ellipse phantoms.

Seeds per workload id ``cid``: phantom 1000+cid, motion 2000+cid,
noise 3000+cid, gate draw 4000+cid+run.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "SLICE_SIDES", "slice_batch", "phantom", "disc_area_image", "rigid_motion",
    "rbf_fields", "noise", "seeds", "random_image", "random_sinogram",
]


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: geometry, gates, motion kind and phantom."""

    name: str
    cid: int                 # workload id, fixes the seeds
    n: int                   # image side (n x n pixels, unit spacing)
    n_angles: int            # parallel-beam angles k*pi/n_angles, k < n_angles
    n_bins: int              # detector bins at unit spacing
    n_gates: int             # N, number of motion states
    motion: str              # "rigid" or "rbf"
    max_rot_deg: float = 0.0     # rigid: rotation U[-max, max] degrees
    max_shift: float = 0.0       # rigid: shift U[-max, max] px per axis
    rbf_count: int = 16          # rbf: Gaussian bumps per field
    rbf_width: float = 40.0      # rbf: Gaussian sigma in px
    rbf_max_disp: float = 8.0    # rbf: max |u(p)| in px after scaling
    n_ellipses: int = 10
    axis_lo: float = 5.0         # ellipse semi-axes U[axis_lo, axis_hi] px
    axis_hi: float = 40.0
    alpha: float = 1e-2          # weight of g(x) = alpha ||x||^2
    epochs: int = 50
    noise_level: float = 0.01    # sigma = level * max clean sinogram value

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)


WORKLOADS = {
    # rigid, FP64 oracle scale: 128^2, 180 angles x 183 bins, N=4
    "rigid128": Workload("rigid128", 1, 128, 180, 183, 4, "rigid",
                         max_rot_deg=5.0, max_shift=3.0, n_ellipses=10,
                         alpha=1e-2, epochs=50),
    # rigid, headline size: 512^2, 720 angles x 729 bins, N=10
    "rigid512": Workload("rigid512", 2, 512, 720, 729, 10, "rigid",
                         max_rot_deg=8.0, max_shift=6.0, n_ellipses=40,
                         alpha=1e-3, epochs=100),
    # non-rigid: 512^2, N=20 fields of 16 Gaussian bumps, max |u| = 8 px
    "rbf512": Workload("rbf512", 3, 512, 720, 729, 20, "rbf",
                       n_ellipses=40, alpha=1e-3, epochs=100),
    # non-rigid, mid size: 256^2, 360 x 365, N=8
    "rbf256": Workload("rbf256", 4, 256, 360, 365, 8, "rbf",
                       n_ellipses=20, alpha=1e-3, epochs=50),
}


SLICE_SIDES = (256, 384, 512, 768, 1024)


def slice_batch(count: int, seed: int = 5000, sides=SLICE_SIDES) -> list:
    """Independent slices of mixed size for batched runs: side drawn from
    `sides` (cycled, so every size appears), angles round(1.4 side), bins
    side + 17, gate count U{4..32}, motion alternating rigid (+-8 deg, +-6 px)
    and dense fields (16 bumps, sigma side/12.8, max |u| = 8 px), 10-40
    ellipses scaled with the side, alpha = 1e-3.  Slice j has workload id
    seed + j (its seeds() follow from it)."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        side = int(sides[j % len(sides)])
        gates = int(rng.integers(4, 33))
        kind = "rigid" if j % 2 == 0 else "rbf"
        out.append(Workload(f"slice{j}_{side}", seed + j, side, int(round(1.4 * side)), side + 17, gates,
                            kind, max_rot_deg=8.0, max_shift=6.0, rbf_width=side / 12.8,
                            n_ellipses=max(10, side // 25), axis_lo=side / 100.0, axis_hi=side / 12.8,
                            alpha=1e-3, epochs=100))
    return out


def seeds(cid: int, run: int = 0) -> dict:
    return {"phantom": 1000 + cid, "motion": 2000 + cid,
            "noise": 3000 + cid, "gates": 4000 + cid + run}


def phantom(n: int, n_ellipses: int, seed: int, axis_lo: float = 5.0,
            axis_hi: float = 40.0) -> np.ndarray:
    """Additive random-ellipse phantom, float64 (n, n), row-major [row, col].

    Centres uniform in the disc of radius 0.35 n about the image centre,
    semi-axes U[axis_lo, axis_hi], orientation U[0, pi), intensity U[0, 1];
    a pixel belongs to an ellipse when its centre does.
    """
    rng = np.random.default_rng(seed)
    h = 0.5 * (n - 1)
    c = np.arange(n) - h
    X, Y = np.meshgrid(c, c)           # X varies along columns, Y along rows
    img = np.zeros((n, n))
    for _ in range(n_ellipses):
        rad = 0.35 * n * np.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = rad * np.cos(ang), rad * np.sin(ang)
        a, b = rng.uniform(axis_lo, axis_hi, size=2)
        psi = rng.uniform(0.0, np.pi)
        val = rng.uniform(0.0, 1.0)
        dx, dy = X - cx, Y - cy
        u = (dx * np.cos(psi) + dy * np.sin(psi)) / a
        v = (-dx * np.sin(psi) + dy * np.cos(psi)) / b
        img[u * u + v * v <= 1.0] += val
    return img


def disc_area_image(n: int, radius: float, supersample: int = 16) -> np.ndarray:
    """Centred disc of the given radius as per-pixel covered area (float64).

    Each pixel is split into supersample^2 sub-pixels whose centres are
    tested for inclusion; the pixel value is the covered fraction.
    """
    h = 0.5 * (n - 1)
    s = supersample
    off = (np.arange(s) + 0.5) / s - 0.5
    c = np.arange(n) - h
    sub = (c[:, None] + off[None, :]).reshape(-1)      # n*s sub-centres
    X, Y = np.meshgrid(sub, sub)
    inside = (X * X + Y * Y <= radius * radius).astype(np.float64)
    return inside.reshape(n, s, n, s).mean(axis=(1, 3))


def rigid_motion(n_gates: int, max_rot_deg: float, max_shift: float,
                 seed: int) -> np.ndarray:
    """Rigid motion per gate, float64 (N, 3) = [phi (rad), tx, ty]; gate 0 = 0."""
    rng = np.random.default_rng(seed)
    m = np.zeros((n_gates, 3))
    if n_gates > 1:
        m[1:, 0] = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, n_gates - 1))
        m[1:, 1:] = rng.uniform(-max_shift, max_shift, (n_gates - 1, 2))
    return m


def rbf_fields(n: int, n_gates: int, seed: int, count: int = 16,
               width: float = 40.0, max_disp: float = 8.0) -> np.ndarray:
    """Dense displacement fields, float32 (N, 2, n, n); gate 0 = 0.

    Channel 0 is the column (x) displacement, channel 1 the row (y)
    displacement, both in pixels.  Each field is a sum of ``count``
    Gaussian bumps of standard deviation ``width`` px with seeded centres
    (uniform over the image) and N(0, I_2) amplitudes, scaled so that the
    largest displacement length over the image equals ``max_disp``.
    """
    rng = np.random.default_rng(seed)
    f = np.zeros((n_gates, 2, n, n), dtype=np.float32)
    idx = np.arange(n, dtype=np.float64)
    C, R = np.meshgrid(idx, idx)
    for g in range(1, n_gates):
        cen = rng.uniform(0.0, n - 1.0, size=(count, 2))   # (col, row)
        amp = rng.standard_normal((count, 2))
        ux = np.zeros((n, n))
        uy = np.zeros((n, n))
        for j in range(count):
            e = np.exp(-((C - cen[j, 0]) ** 2 + (R - cen[j, 1]) ** 2)
                       / (2.0 * width * width))
            ux += amp[j, 0] * e
            uy += amp[j, 1] * e
        mag = np.sqrt(ux * ux + uy * uy).max()
        scale = max_disp / mag if mag > 0 else 0.0
        f[g, 0] = (ux * scale).astype(np.float32)
        f[g, 1] = (uy * scale).astype(np.float32)
    return f


def noise(n_gates: int, n_angles: int, n_bins: int, seed: int) -> np.ndarray:
    """Standard normal draws, float64 (N, n_angles, n_bins)."""
    return np.random.default_rng(seed).standard_normal((n_gates, n_angles, n_bins))


def random_image(n: int, seed: int) -> np.ndarray:
    """U[0,1) test image, float64 (n, n)."""
    return np.random.default_rng(seed).uniform(size=(n, n))


def random_sinogram(n_angles: int, n_bins: int, seed: int) -> np.ndarray:
    """Standard normal test sinogram, float64 (n_angles, n_bins)."""
    return np.random.default_rng(seed).standard_normal((n_angles, n_bins))
