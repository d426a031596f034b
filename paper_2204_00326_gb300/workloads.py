"""Seeded synthetic inputs: contrast functions, incident waves, random vectors.

This module holds none of the method's arithmetic.  It only produces the data
both the CUDA path and the test oracle consume, so both read identical inputs.
The shapes follow the paper's experiments (Section 6): a Gaussian contrast
(Eq. gaussianContrast), mixtures of Gaussian bumps like Experiment 7, a
discontinuous disc standing in for the cavity/lens contrasts of Experiments
8-9, and plane waves ``exp(i kappa (x cos t + y sin t))``.

Random draws use numpy's PCG64 with an explicit seed; for a bump mixture the
order is centres, then widths, then amplitudes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: grid, wavenumber, contrast and right-hand sides."""

    name: str
    n_side: int            # grid points per side (p * leaves per side)
    kappa: float
    contrast: str          # "gauss_trunc" | "bumps" | "disc"
    nbumps: int = 0
    seed: int = 0
    nrhs: int = 1
    tol: float = 1e-8
    x0: float = -1.0
    x1: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n_side * self.n_side


# The five workloads (uniform p = 4 grids on [-1, 1]^2).
GRID32_K8 = Workload("grid32_k8_gauss", 32, 8.0, "gauss_trunc", tol=1e-10)
GRID128_K40 = Workload("grid128_k40_bumps4", 128, 40.0, "bumps", nbumps=4, seed=0)
GRID256_K80 = Workload("grid256_k80_disc", 256, 80.0, "disc", nrhs=64)
GRID512_K160 = Workload("grid512_k160_bumps8", 512, 160.0, "bumps", nbumps=8, seed=1)
# Experiment 1 (Section 6.2): point charges at the Chebyshev nodes of a uniform
# grid on [-1,1]^2, kappa = 50, random charges; the paper uses p = 10 nodes per
# leaf side on 32 x 32 leaves (N = 102400), the library p = 4 on 64 x 64
# leaves (N = 65536, leaf kappa w = 0.78, low frequency as in the paper).
NBODY256_K50 = Workload("nbody256_k50", 256, 50.0, "zero")
WORKLOADS = {w.name: w for w in (GRID32_K8, GRID128_K40, GRID256_K80, GRID512_K160)}


def mixed_size_batch(count: int = 16, sizes=(64, 128, 256, 512, 1024), seed: int = 5, nrhs: int = 8) -> list:
    """The mixed-size batch of problems: grids drawn from `sizes`, kappa =
    0.3 sqrt(N) (the same points per wavelength at every size), contrast a
    Gaussian-bump mixture (as in the 128^2 workload, 4 bumps) or the disc,
    each with probability 1/2, all from one seed; nrhs plane waves each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        n = int(sizes[rng.integers(len(sizes))])
        if rng.random() < 0.5:
            out.append(Workload(f"batch{k}_grid{n}_bumps4", n, 0.3 * n, "bumps", nbumps=4, seed=seed * 1000 + k, nrhs=nrhs))
        else:
            out.append(Workload(f"batch{k}_grid{n}_disc", n, 0.3 * n, "disc", nrhs=nrhs))
    return out


def contrast(w: Workload, xy: np.ndarray) -> np.ndarray:
    """q(x) at the points xy (N x 2)."""
    x, y = xy[:, 0], xy[:, 1]
    r2 = x * x + y * y
    if w.contrast == "gauss_trunc":
        return np.where(r2 <= 0.81, 1.5 * np.exp(-16.0 * r2), 0.0)
    if w.contrast == "zero":
        return np.zeros(len(x))
    if w.contrast == "disc":
        return np.where(r2 < 0.25, 2.0, 0.0)
    if w.contrast == "bumps":
        rng = np.random.Generator(np.random.PCG64(w.seed))
        centres = rng.uniform(-0.6, 0.6, size=(w.nbumps, 2))
        widths = rng.uniform(0.1, 0.3, size=w.nbumps)
        amps = rng.uniform(0.5, 2.0, size=w.nbumps)
        q = np.zeros(len(x))
        for c, s, a in zip(centres, widths, amps):
            q += a * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / (s * s))
        return q
    raise ValueError(f"unknown contrast {w.contrast!r}")


def plane_waves(kappa: float, xy: np.ndarray, nrhs: int = 1) -> np.ndarray:
    """u_inc for nrhs directions theta_k = 2 pi k / nrhs, shape (N, nrhs)."""
    th = 2.0 * np.pi * np.arange(nrhs) / nrhs
    ph = xy[:, 0:1] * np.cos(th)[None, :] + xy[:, 1:2] * np.sin(th)[None, :]
    return np.exp(1j * kappa * ph)


def random_vector(N: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """Complex standard-normal test vectors, shape (N, nrhs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((N, nrhs)) + 1j * rng.standard_normal((N, nrhs))
