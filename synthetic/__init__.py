"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws and shapes input fields (initial mole fractions and
binary Maxwell-Stefan diffusivities).  It holds none of the lattice Boltzmann
arithmetic: no equilibria, no relaxation matrices, no streaming.  Both sides
of every parity test read the arrays it returns, so they see identical data.

All arrays are float64, laid out species-major: ``x0[sigma, z, y, x]`` (2D
fields use ``nz == 1``).  Every field is renormalised so that the N mole
fractions sum to one at each node (Sec. 2, Eq. 2-3b of the paper).

Recipes (lattice units, cell centres at integer index + 1/2):

* ``sin_modes``      -- per species one Fourier mode of amplitude ``amp`` with a
  seeded wave vector in {1..4}^2 and a seeded phase, on a uniform 1/N base.
* ``two_bulb``       -- a tanh interface of width ``width`` cells along x
  between a left and a right composition (Loschmidt-tube / two-bulb shape).
* ``gaussian_blobs`` -- ``nblobs`` periodic Gaussian blobs per species
  (minimum-image distance) of width ``sigma`` and amplitude ``amp`` added to a
  uniform 1/N background.
* ``random_D``       -- symmetric binary diffusivities uniform in [lo, hi].
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng",
    "renormalise",
    "sin_modes",
    "two_bulb",
    "gaussian_blobs",
    "random_D",
    "D_from_pairs",
    "duncan_toor_1d",
    "loschmidt_1d",
    "small_mode",
    "batch_instances",
    "batch_field",
    "erf_step",
]


def rng(seed: int) -> np.random.Generator:
    """NumPy PCG64 generator for one workload seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def renormalise(x: np.ndarray) -> np.ndarray:
    """Scale the N species so that they sum to one at every node."""
    s = x.sum(axis=0, keepdims=True)
    return x / s


def sin_modes(N: int, nx: int, ny: int, nz: int = 1, *, amp: float = 0.05,
              seed: int = 1001) -> np.ndarray:
    """One seeded sinusoidal mode per species on a 1/N background, renormalised."""
    g = rng(seed)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5,
                          np.arange(nx) + 0.5, indexing="ij")
    out = np.empty((N, nz, ny, nx))
    for s in range(N):
        kx, ky = g.integers(1, 5, size=2)
        kz = g.integers(1, 5) if nz > 1 else 0
        phi = g.uniform(0.0, 2.0 * math.pi)
        arg = 2.0 * math.pi * (kx * x / nx + ky * y / ny + (kz * z / nz if nz > 1 else 0.0)) + phi
        out[s] = 1.0 / N + amp * np.sin(arg)
    return renormalise(out)


def two_bulb(nx: int, ny: int, nz: int, *, left=(0.0, 0.5, 0.5),
             right=(0.5, 0.5, 0.0), width: float = 4.0) -> np.ndarray:
    """Two compositions joined by a tanh interface of ``width`` cells at nx/2."""
    left = np.asarray(left, dtype=np.float64)
    right = np.asarray(right, dtype=np.float64)
    X = np.arange(nx) + 0.5
    h = 0.5 * (1.0 + np.tanh((X - nx / 2.0) / width))
    prof = left[:, None] + (right - left)[:, None] * h[None, :]
    out = np.broadcast_to(prof[:, None, None, :], (left.size, nz, ny, nx)).copy()
    return renormalise(out)


def gaussian_blobs(N: int, nx: int, ny: int, *, nblobs: int = 8, sigma: float = 32.0,
                   amp: float = 0.2, seed: int = 1003) -> np.ndarray:
    """Seeded periodic Gaussian blobs per species on a uniform 1/N background."""
    g = rng(seed)
    y, x = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    out = np.full((N, 1, ny, nx), 1.0 / N)
    for s in range(N):
        cx = g.uniform(0.0, nx, size=nblobs)
        cy = g.uniform(0.0, ny, size=nblobs)
        for b in range(nblobs):
            dx = np.abs(x - cx[b])
            dx = np.minimum(dx, nx - dx)
            dy = np.abs(y - cy[b])
            dy = np.minimum(dy, ny - dy)
            out[s, 0] += amp * np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
    return renormalise(out)


def random_D(N: int, *, lo: float = 0.01, hi: float = 0.12, seed: int = 1003) -> np.ndarray:
    """Symmetric N x N binary diffusivities uniform in [lo, hi]; diagonal set to 1."""
    g = rng(seed)
    D = np.ones((N, N))
    for i in range(N):
        for j in range(i + 1, N):
            D[i, j] = D[j, i] = g.uniform(lo, hi)
    return D


def D_from_pairs(N: int, pairs: dict) -> np.ndarray:
    """Build a symmetric N x N matrix from {(i, j): D_ij} with 1-based species."""
    D = np.ones((N, N))
    for (i, j), v in pairs.items():
        D[i - 1, j - 1] = D[j - 1, i - 1] = float(v)
    return D


def duncan_toor_1d(nx: int) -> np.ndarray:
    """Ternary initial field of the Duncan-Toor-like problem (Sec. 4.2) on [0, 1].

    xi_1 is 0.8 below x = 0.25, falls linearly as 1.6 (0.75 - x) to zero at
    x = 0.75, and is zero above; xi_2 = 0.2 everywhere; xi_3 closes the sum.
    """
    X = (np.arange(nx) + 0.5) / nx
    x1 = np.where(X < 0.25, 0.8, np.where(X < 0.75, 1.6 * (0.75 - X), 0.0))
    x2 = np.full(nx, 0.2)
    x3 = 1.0 - x1 - x2
    return np.stack([x1, x2, x3])[:, None, None, :].copy()


def loschmidt_1d(n: int) -> np.ndarray:
    """Ternary Loschmidt-tube initial field (Sec. 4.3) along a tube of n cells.

    The first half (bottom) holds (0, 0.509, 0.491), the second half (top)
    holds (0.515, 0.485, 0).
    """
    out = np.empty((3, 1, 1, n))
    bottom = np.array([0.0, 0.509, 0.491])
    top = np.array([0.515, 0.485, 0.0])
    out[:, 0, 0, : n // 2] = bottom[:, None]
    out[:, 0, 0, n // 2:] = top[:, None]
    return out


def small_mode(xbar, vec, eps: float, nx: int, ny: int = 1, nz: int = 1, *,
               k=(1, 0, 0)) -> np.ndarray:
    """Uniform composition ``xbar`` plus ``eps * vec * cos(2 pi k . X / n)``.

    ``vec`` has N entries summing to zero, so the field still sums to one.
    """
    xbar = np.asarray(xbar, dtype=np.float64)
    vec = np.asarray(vec, dtype=np.float64)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2.0 * math.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz)
    return xbar[:, None, None, None] + eps * vec[:, None, None, None] * np.cos(ph)[None]


def batch_instances(count: int, *, lo: int = 32, hi: int = 256, seed: int = 1004,
                    d_lo: float = 0.01, d_hi: float = 0.12):
    """Uneven ternary D2Q5 instances: square side L uniform in [lo, hi], seeded
    diffusivities uniform in [d_lo, d_hi]; even instances get one sine mode per
    species on a periodic grid, odd instances the two-bulb tanh profile along x
    with no-flux x faces and periodic y.

    Returns (grids[count, 3], D[count, 3, 3], bcs: list of count 6-tuples); the
    initial fields come one at a time from ``batch_field(i, L_i)``.
    """
    g = rng(seed)
    sides = g.integers(lo, hi + 1, size=count)
    grids = np.stack([sides, sides, np.ones_like(sides)], axis=1).astype(np.int32)
    Ds = np.empty((count, 3, 3))
    for i in range(count):
        d12, d13, d23 = g.uniform(d_lo, d_hi, size=3)
        Ds[i] = D_from_pairs(3, {(1, 2): d12, (1, 3): d13, (2, 3): d23})
    P, W = "periodic", "noflux"
    bcs = [(P,) * 6 if i % 2 == 0 else (W, W, P, P, P, P) for i in range(count)]
    return grids, Ds, bcs


def batch_field(i: int, side: int, *, seed: int = 1004) -> np.ndarray:
    """Initial field of instance i of ``batch_instances`` (see there)."""
    if i % 2 == 0:
        return sin_modes(3, side, side, amp=0.05, seed=seed * 7919 + i)
    return two_bulb(side, side, 1, width=4.0)


def erf_step(nx: int, ny: int = 1, *, C0: float = 0.9, C1: float = 0.1,
             half_width: float = 6.0) -> np.ndarray:
    """Binary step of Sec. 4.1 on [-half_width, half_width] (cell centres):
    xi_1 = C0 for x < 0 and C1 for x >= 0, xi_2 = 1 - xi_1."""
    dx = 2.0 * half_width / nx
    X = -half_width + (np.arange(nx) + 0.5) * dx
    x1 = np.where(X < 0.0, C0, C1)
    out = np.empty((2, 1, ny, nx))
    out[0] = x1[None, None, :]
    out[1] = 1.0 - out[0]
    return out
