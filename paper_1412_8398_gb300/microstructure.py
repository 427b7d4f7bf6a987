"""Seeded synthetic inputs: phase images and per-phase moduli.

This module only *builds inputs*. It holds none of the method's arithmetic
(no Green operator, no transform, no scheme), so both the CUDA path and the
CPU oracle can take their inputs from it without sharing any solver code.

Conventions
-----------
* A phase image is a ``uint8`` numpy array.  In 3D its shape is
  ``(n3, n2, n1)`` and in 2D ``(n2, n1)``: C order, so x1 (``n1``) is the
  fastest-varying index, which is the layout the C ABI expects.
* Voxel centres sit at integer coordinates ``0 .. n-1`` along every axis.
* Phase 0 is the matrix and phase 1 the inclusions (the paper's phases 1 and
  2, Sec. 2).

Random numbers come from SplitMix64 (Steele, Lea and Flood 2014), written
out here so that every platform draws the same sequence for a given seed.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "SplitMix64",
    "boolean_spheres",
    "batch_recipe",
    "centered_disc",
    "square_inclusion",
    "laminate",
    "periodic_sphere",
    "lame_from_young",
    "binary_moduli",
    "young_poisson_phases",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64: output i is mix(seed + (i + 1) * golden)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + n + 1, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            z = self.state + idx * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles uniform in [0, 1): the top 53 bits of each output."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def poisson(self, lam: float) -> int:
        """Poisson(lam) by counting unit-rate exponential arrivals in [0, lam]."""
        if lam <= 0.0:
            return 0
        total = 0.0
        count = 0
        chunk = int(lam + 10.0 * math.sqrt(lam) + 16)
        while True:
            u = self.uniform(chunk)
            gaps = -np.log1p(-u)
            csum = total + np.cumsum(gaps)
            inside = int(np.searchsorted(csum, lam, side="right"))
            count += inside
            if inside < chunk:
                return count
            total = float(csum[-1])


def _voxelize_balls(shape_xyz, centers, radius):
    """Mark every voxel whose centre lies within `radius` of a centre, periodically."""
    d = len(shape_xyz)
    img = np.zeros(tuple(reversed(shape_xyz)), dtype=np.uint8)  # numpy order: (.., x2, x1)
    r2 = radius * radius
    for c in centers:
        axes = []
        for i in range(d):
            lo = math.ceil(c[i] - radius)
            hi = math.floor(c[i] + radius)
            coords = np.arange(lo, hi + 1)
            axes.append(coords)
        # squared distances on the (unwrapped) bounding box
        grids = np.meshgrid(*[(a - c[i]) ** 2 for i, a in enumerate(axes)], indexing="ij")
        dist2 = sum(grids)
        inside = dist2 <= r2
        idx = np.nonzero(inside)
        wrapped = [np.mod(axes[i][idx[i]], shape_xyz[i]) for i in range(d)]
        img[tuple(reversed(wrapped))] = 1
    return img


def boolean_spheres(shape, radius: float, fraction: float, seed: int):
    """Periodised Boolean model of balls (Poisson centres), Sec. 6.1 microstructure.

    shape: (n1, n2, n3) in 3D or (n1, n2) in 2D (x1 first).
    The intensity is chosen so that the expected inclusion fraction is
    `fraction`: theta = -ln(1 - f) / |ball| per voxel; the count is
    Poisson(theta N) and the centres are uniform in [0, n)^d.
    Returns (phase image, info) where info records the seed, the number of
    centres and the realised fraction.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    n_vox = int(np.prod(shape))
    vol = (4.0 / 3.0) * math.pi * radius**3 if d == 3 else math.pi * radius**2
    theta = -math.log(1.0 - fraction) / vol
    rng = SplitMix64(seed)
    count = rng.poisson(theta * n_vox)
    u = rng.uniform(count * d).reshape(count, d) if count else np.zeros((0, d))
    centers = u * np.asarray(shape, dtype=np.float64)
    img = _voxelize_balls(shape, centers, radius)
    info = {
        "seed": seed,
        "n_centers": count,
        "radius": radius,
        "target_fraction": fraction,
        "fraction": float(img.mean()),
    }
    return img, info


def centered_disc(n: int, fraction: float):
    """2D n x n image with one disc of area fraction `fraction` at the centre.

    The centre is ((n-1)/2, (n-1)/2) and the radius n*sqrt(f/pi); a pixel is
    inclusion (1) iff its centre lies within the radius.  The image is
    symmetric under x <-> y and under (x, y) -> (n-1-x, n-1-y).
    """
    r = n * math.sqrt(fraction / math.pi)
    c = (n - 1) / 2.0
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return (((x - c) ** 2 + (y - c) ** 2) <= r * r).astype(np.uint8)


def square_inclusion(n: int, dim: int = 2):
    """n^d image with a centred square (cube) inclusion of side n/2 (n even)."""
    lo, hi = n // 4, n // 4 + n // 2
    img = np.zeros((n,) * dim, dtype=np.uint8)
    img[(slice(lo, hi),) * dim] = 1
    return img


def laminate(shape, layers_x1):
    """Phase varies along x1 only: voxel (x1, ...) gets phase layers_x1[x1]."""
    shape = tuple(int(s) for s in shape)
    layers = np.asarray(layers_x1, dtype=np.uint8)
    assert layers.shape == (shape[0],)
    img = np.empty(tuple(reversed(shape)), dtype=np.uint8)
    img[...] = layers  # broadcast along the last (x1) axis
    return img


def periodic_sphere(n: int, fraction: float):
    """n^3 image with one centred ball of volume fraction `fraction` (Sec. 5.3)."""
    r = n * (3.0 * fraction / (4.0 * math.pi)) ** (1.0 / 3.0)
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) <= r * r).astype(np.uint8)


def lame_from_young(E: float, nu: float):
    """Lame coefficients (lambda, mu) from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def young_poisson_phases(pairs):
    """Per-phase (lambda, mu) arrays from a list of (E, nu) pairs."""
    lm = [lame_from_young(E, nu) for E, nu in pairs]
    return (np.array([a for a, _ in lm], dtype=np.float64),
            np.array([b for _, b in lm], dtype=np.float64))


def binary_moduli(chi: float, dim: int):
    """The paper's binary medium (Sec. 2): kappa1 = 1, mu1 = 0.6, phase 2 = chi x phase 1.

    lambda1 = 0.4 in 2D and 0.6 in 3D (kappa = lambda + (2/d) mu).
    """
    lam1 = 0.4 if dim == 2 else 0.6
    mu1 = 0.6
    return (np.array([lam1, chi * lam1], dtype=np.float64),
            np.array([mu1, chi * mu1], dtype=np.float64))


BATCH_LENGTHS = (32, 48, 64, 96, 128)


def batch_recipe(count: int, first_seed: int = 1000, lengths=BATCH_LENGTHS):
    """Parameters of `count` independent Boolean-sphere samples of uneven sizes.

    Sample s (seed first_seed + s) draws, from SplitMix64 seeded with its seed:
    the grid length L uniformly from `lengths` (cubic grid), the sphere radius
    uniformly in [3, 8] voxels, the target inclusion fraction uniformly in
    [0.1, 0.4] and the stiffness contrast E_incl / E_matrix log-uniformly in
    [10, 1000] (nu = 0.3 in both phases, E_matrix = 1).  The microstructure itself
    is ``boolean_spheres((L, L, L), radius, fraction, seed)``.
    Returns a list of dicts with keys seed, L, radius, fraction, contrast.
    """
    out = []
    for s in range(count):
        seed = first_seed + s
        u = SplitMix64(seed ^ 0x5A5A5A5A).uniform(4)
        L = int(lengths[min(int(u[0] * len(lengths)), len(lengths) - 1)])
        out.append({"seed": seed, "L": L, "radius": 3.0 + 5.0 * float(u[1]),
                    "fraction": 0.1 + 0.3 * float(u[2]), "contrast": float(10.0 ** (1.0 + 2.0 * u[3]))})
    return out


def batch_sample(spec):
    """Phase image and (lambda, mu) of one sample of ``batch_recipe``."""
    L = spec["L"]
    ph, info = boolean_spheres((L, L, L), spec["radius"], spec["fraction"], spec["seed"])
    lam, mu = young_poisson_phases([(1.0, 0.3), (spec["contrast"], 0.3)])
    return ph, lam, mu, info
