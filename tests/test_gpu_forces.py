"""The chemical potentials and forces of the fused step's thermodynamics
(lbm_forces) against the binary64 oracle.

mu_i = RT ln f_i - sqrt(kappa_i) lap psi (Eqs. 4-6, 9-12) and F_i = -rho~_i
grad mu_i (Eq. 5).  The oracle's F is its literal Eq. (5) (double sum over
kappa_ij); its mu is its ln f_i times RT minus sqrt(kappa_i) times its
lattice Laplacian of psi.

Tolerances:
* binary64 (LBM_FP64): mu within 1e-13 of max |mu_i|, F within 1e-12 of
  max |F_i| (rounding order only).
* double-binary32 (LBM_FP32DEV fused): mu carries about 2^-44 of its
  largest term, so |mu - mu_orc| <= 2^-42 max |mu_i| (a factor 4 of
  margin).  Each gradient difference mu(r + e) - mu(r - e) is taken on the
  (hi, lo) pairs and rounded once to binary32, so it is exact to 2^-24 of
  itself plus the df64 error of mu; the stencil then sums the differences in
  binary32.  So |F - F_orc| <= rho~_i (2^-21 S + 2^-40 max |mu_i|) + 2^-22
  |F_orc|, with S = 3 (|d_E| / 9 + (|d_NE| + |d_SE|) / 36) the stencil's
  absolute terms (x; y likewise), which the binary32 sum can lose when they
  cancel.  S is the size of the local differences of mu, so binary32
  thermodynamics (LBM_FP32, mu within 2^-21 of max |mu_i|, far larger than
  S) misses the bound by orders of magnitude, which the test also checks:
  the test tells the two arithmetic forms apart.
"""
from __future__ import annotations

import numpy as np
import pytest

from helpers import gpu_problem, oracle_problem, seeded_mixture, smooth_rho
from paper_2306_10652_gb300 import synth

pytestmark = pytest.mark.gpu

FP64, FP32DEV, FP32 = 0, 1, 2

CASES = [
    # seed, nc, shape, random M, density range
    (201, 2, (1, 37, 250), True, (0.05, 0.6)),
    (202, 3, (1, 64, 64), False, (0.02, 0.7)),
    (203, 10, (1, 40, 130), True, (0.05, 0.5)),
    (204, 16, (1, 9, 131), False, (0.05, 0.4)),
]


def oracle_fields(c, shape, M, rho):
    orc = oracle_problem(c, 0, shape, M=M)
    mo = orc.moments(orc.init_equilibrium(rho))
    kappa = 0.02 * np.asarray(c["a"]) / c["a"][0]                       # Eq. (6)
    rm = rho / (np.ones(len(c["a"])) if M is None else M)[:, None, None, None]
    psi = (np.sqrt(kappa)[:, None, None, None] * rm).sum(axis=0)        # Eq. (4)
    lap = orc.laplacian(psi)
    RT = orc.R * orc.T
    mu = RT * mo["lnf"] - np.sqrt(kappa)[:, None, None, None] * lap[None]
    return mu, mo["F"], rm


def stencil_abs(m):
    """Absolute terms of the D2Q9 gradient stencil of m[nz, ny, nx]: (S_x, S_y)."""
    sh = lambda dx, dy: np.roll(m, shift=(-dy, -dx), axis=(-2, -1))
    dE = np.abs(sh(1, 0) - sh(-1, 0))
    dN = np.abs(sh(0, 1) - sh(0, -1))
    dNE = np.abs(sh(1, 1) - sh(-1, -1))
    dSE = np.abs(sh(1, -1) - sh(-1, 1))
    return np.stack([3 * (dE / 9 + (dNE + dSE) / 36), 3 * (dN / 9 + (dNE + dSE) / 36)])


def run(case, precision):
    seed, nc, shape, Mr, (lo, hi) = case
    c = seeded_mixture(seed, nc, 0, shape)
    M = synth.uniform(seed, 0.5, 2.0, nc) if Mr else None
    rho = smooth_rho(seed, c, shape, lo, hi) * (1.0 if M is None else M[:, None, None, None])
    with gpu_problem(c, 0, shape, M=M, precision=precision, schedule=2) as gp:
        gp.init_fields(rho)
        exact = gp.moments(("rho",))["rho"]       # the densities the state holds
        out = gp.forces()
    mu_o, F_o, rm = oracle_fields(c, shape, M, exact)
    return out["mu"], out["F"], mu_o, F_o, rm


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nc{c[1]}-{c[2][1]}x{c[2][2]}")
def test_forces_binary64(case):
    mu, F, mu_o, F_o, _ = run(case, FP64)
    for i in range(mu.shape[0]):
        assert np.abs(mu[i] - mu_o[i]).max() <= 1e-13 * np.abs(mu_o[i]).max()
        assert np.abs(F[i] - F_o[i]).max() <= 1e-12 * np.abs(F_o[i]).max()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nc{c[1]}-{c[2][1]}x{c[2][2]}")
def test_forces_double_binary32(case):
    mu, F, mu_o, F_o, rm = run(case, FP32DEV)
    for i in range(mu.shape[0]):
        mscale = np.abs(mu_o[i]).max()
        assert np.abs(mu[i] - mu_o[i]).max() <= 2.0 ** -42 * mscale, \
            (i, np.abs(mu[i] - mu_o[i]).max() / mscale)
        S = stencil_abs(mu_o[i])
        bound = rm[i][None] * (2.0 ** -21 * S + 2.0 ** -40 * mscale) + 2.0 ** -22 * np.abs(F_o[i])
        assert (np.abs(F[i] - F_o[i]) <= bound).all(), (i, (np.abs(F[i] - F_o[i]) / bound).max())


def test_binary32_thermodynamics_is_distinguishable():
    """LBM_FP32 misses the double-binary32 bounds on mu and F by wide margins."""
    mu, F, mu_o, F_o, rm = run(CASES[2], FP32)
    ratio = max(np.abs(mu[i] - mu_o[i]).max() / (2.0 ** -42 * np.abs(mu_o[i]).max()) for i in range(mu.shape[0]))
    assert ratio > 1e3, ratio
    fr = 0.0
    for i in range(mu.shape[0]):
        bound = rm[i][None] * (2.0 ** -21 * stencil_abs(mu_o[i]) + 2.0 ** -40 * np.abs(mu_o[i]).max()) \
            + 2.0 ** -22 * np.abs(F_o[i])
        fr = max(fr, (np.abs(F[i] - F_o[i]) / bound).max())
    assert fr > 10, fr
