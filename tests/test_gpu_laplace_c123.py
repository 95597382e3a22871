"""The Young-Laplace check of Sec. 3.1 with the paper's own mixture (binary32
throughout, LBM_FP32): C1, C2 and C3 at 250 K, the flash of z = (0.5, 0.25,
0.25) at 50 bar (Eq. 13 start, W = 4), 200 x 200, tau = 1, delta = 0, lattice
units from R = 1, a_C1 = 2/49, b_C1 = 2/21, M_C1 = 1, C1 the reference of Eq.
(6); radii 20, 30, 40, 50; 2e5 steps (the paper runs 1e6; the jumps move by
under 2.5 % between the two).

* For kappa_ref = 0.02 and 0.04 the pressure jump dp = p(centre) - p(corner)
  is linear in 1/R: R^2 >= 0.999, intercept within 3 % of the largest jump.
* The surface tension (the slope) grows with kappa_ref as in diffuse-interface
  theory (sigma proportional to sqrt(kappa)): the ratio of the two slopes is
  sqrt(2) within 10 %.
The paper also shows kappa_ref = 0.06.  With the isotropic central-difference
stencils (the reading for the unprinted discretisation of grad and lap) this
mixture diverges within a few thousand steps from kappa_ref = 0.05 on, in
binary32 and binary64 alike (C3 gets 4.07 kappa_ref), so it is not run.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle.thermo import LatticeUnits, flash
from oracle.workloads import droplet

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N = 200
RADII = (20, 30, 40, 50)
STEPS = 200000


def mixture():
    comp = {}
    for line in open(f"{GOLDEN}/components.txt"):
        if line.startswith("#") or not line.strip():
            continue
        name, pc, Tc, om, M = line.split()
        comp[name] = (float(pc), float(Tc), float(om), float(M))
    sel = [comp[n] for n in ("C1", "C2", "C3")]
    return LatticeUnits([s[1] for s in sel], [s[0] for s in sel], [s[2] for s in sel], [s[3] for s in sel])


def series(kappa_ref, T=250.0):
    from paper_2306_10652_gb300 import lbmfug
    lu = mixture()
    fl = flash(lu.problem(T), lu.p(50.0), np.array([0.5, 0.25, 0.25]))
    assert fl is not None
    dps = []
    for R in RADII:
        rho = droplet(fl.rhoi_V, fl.rhoi_L, N, N, R)[:, None] * lu.M[:, None, None, None]
        with lbmfug.Problem(0, N, N, 1, lu.a, lu.b, lu.omega, None, lu.T(T), 1.0, M=lu.M, kappa_ref=kappa_ref,
                            precision=2) as gp:
            gp.init_fields(rho)
            gp.step(STEPS)
            p = gp.moments(("p",))["p"][0]
        dps.append(p[N // 2, N // 2] - p[0, 0])
    x = 1.0 / np.array(RADII, float)
    y = np.array(dps)
    A = np.vstack([x, np.ones_like(x)]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, y, rcond=None)
    fit = A @ np.array([slope, icpt])
    r2 = 1.0 - ((y - fit) ** 2).sum() / ((y - y.mean()) ** 2).sum()
    return {"dp": y, "slope": slope, "icpt": icpt, "r2": r2}


@pytest.fixture(scope="module")
def fits():
    return {k: series(k) for k in (0.02, 0.04)}


@pytest.mark.parametrize("kappa_ref", [0.02, 0.04])
def test_laplace_linear(fits, kappa_ref):
    f = fits[kappa_ref]
    assert np.isfinite(f["dp"]).all() and (f["dp"] > 0).all(), f["dp"]
    assert f["r2"] >= 0.999, f
    assert abs(f["icpt"]) <= 0.03 * f["dp"].max(), f


def test_surface_tension_grows_as_sqrt_kappa(fits):
    ratio = fits[0.04]["slope"] / fits[0.02]["slope"]
    assert abs(ratio / np.sqrt(2.0) - 1.0) <= 0.10, ratio
