"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds random draws only -- no step of the method.  Every
generator takes an explicit seed and uses numpy's PCG64 so that both sides
receive bit-identical inputs.

Recipes (lattice units, R = 1; the reduced parameters scatter around the
paper's C1 reference a = 2/49, b = 2/21 of Sec. 3.1):

* ``pr_components``: a_i = 2/49 * U[a_lo, a_hi], b_i = 2/21 * U[b_lo, b_hi],
  omega_i ~ U[0, 0.5], symmetric delta_ij ~ U[k_lo, k_hi] with zero diagonal.
* ``dirichlet``: an overall composition z ~ Dirichlet(1, ..., 1).
* ``multiplicative_noise``: 1 + amp * U[-1, 1], independent per node and component.
* ``random_state``: smooth random density fields for step-by-step parity runs.
"""
from __future__ import annotations

import numpy as np

A_C1 = 2.0 / 49.0
B_C1 = 2.0 / 21.0


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def pr_components(seed: int, nc: int, a_range=(0.6, 1.6), b_range=(0.8, 1.2),
                  omega_range=(0.0, 0.5), k_range=(0.0, 0.1)):
    rng = rng_for(seed, 1)
    a = A_C1 * rng.uniform(a_range[0], a_range[1], nc)
    b = B_C1 * rng.uniform(b_range[0], b_range[1], nc)
    omega = rng.uniform(omega_range[0], omega_range[1], nc)
    kij = np.zeros((nc, nc))
    iu = np.triu_indices(nc, 1)
    kij[iu] = rng.uniform(k_range[0], k_range[1], len(iu[0]))
    kij = kij + kij.T
    return {"a": a, "b": b, "omega": omega, "kij": kij}


def dirichlet(seed: int, nc: int, stream: int = 2):
    return rng_for(seed, stream).dirichlet(np.ones(nc))


def uniform(seed: int, lo: float, hi: float, size=None, stream: int = 3):
    return rng_for(seed, stream).uniform(lo, hi, size)


def multiplicative_noise(seed: int, shape, amp: float, stream: int = 4):
    return 1.0 + amp * rng_for(seed, stream).uniform(-1.0, 1.0, shape)


def random_state(seed: int, nc: int, shape, lo=0.05, hi=1.0, modes=3, stream: int = 5):
    """Smooth, strictly positive random fields rho[i, z, y, x] in (lo, hi).

    Built from a few random low Fourier modes per component so that the
    fields have interface-like gradients without any grid-scale noise.
    """
    rng = rng_for(seed, stream)
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.empty((nc,) + tuple(shape))
    for i in range(nc):
        f = np.zeros(shape)
        for _ in range(modes):
            kx, ky, kz = rng.integers(0, 3, 3)
            ph = rng.uniform(0, 2 * np.pi)
            amp = rng.uniform(0.2, 1.0)
            f += amp * np.cos(2 * np.pi * (kx * xx / nx + ky * yy / ny + kz * zz / nz) + ph)
        f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
        out[i] = lo + (hi - lo) * f
    return out


def random_velocity(seed: int, D: int, shape, amp=1e-3, stream: int = 6):
    return amp * rng_for(seed, stream).uniform(-1.0, 1.0, (D,) + tuple(shape))
