"""Physical set-up of the synthetic workloads, computed with the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The random draws come
from ``paper_2306_10652_gb300.synth``; everything that needs the method's
thermodynamics (the flash, the spinodal test) is done here, on the CPU.

* ``two_phase_pressure``: pressure at which the flash of z gives a target
  vapour volume fraction S_V (bisection; S_V falls as p rises).
* ``slab``: Eq. (15) initial profile, vapour-liquid-vapour along x.
* ``droplet``: Eq. (13) initial profile, a liquid disc of radius R.
* ``spinodal_point``: a uniform state inside the spinodal region along the
  line of fixed composition z.
"""
from __future__ import annotations

import numpy as np

from .orc import OracleProblem
from .thermo import flash, min_stability_eigenvalue


def two_phase_interval(P: OracleProblem, z, npts=600, pmin=1e-6, pmax=1.0):
    """(p_lo, p_hi) bracketing the pressures where the flash of z splits."""
    ps = np.geomspace(pmin, pmax, npts)
    ok = [flash(P, p, z) is not None for p in ps]
    idx = [i for i, v in enumerate(ok) if v]
    if not idx:
        return None
    return ps[max(idx[0] - 1, 0)], ps[min(idx[-1] + 1, npts - 1)], ps[idx[0]], ps[idx[-1]]


def two_phase_pressure(P: OracleProblem, z, SV=0.5, tol=1e-10, npts=600):
    """Pressure with flash vapour volume fraction S_V = SV, and the flash there."""
    iv = two_phase_interval(P, z, npts=npts)
    if iv is None:
        return None
    _, _, lo, hi = iv
    rlo, rhi = flash(P, lo, z), flash(P, hi, z)
    if rlo.S_V < SV or rhi.S_V > SV:
        # refine the bracket edges toward the ends of the two-phase range
        return None
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        r = flash(P, mid, z)
        if r is None:
            # the flash may fail very close to the phase boundary: shrink
            hi = mid
            continue
        if r.S_V > SV:
            lo = mid
        else:
            hi = mid
        if hi / lo - 1 < tol:
            break
    p = np.sqrt(lo * hi)
    return p, flash(P, p, z)


def slab(rhoi_V, rhoi_L, nx, SV=0.5, W=4.0):
    """Eq. (15): rho_i(x) for a liquid band in the middle of a periodic box."""
    x = np.arange(nx, dtype=float)
    rv = np.asarray(rhoi_V, float)[:, None]
    rl = np.asarray(rhoi_L, float)[:, None]
    return rv + 0.5 * (rl - rv) * (np.tanh(2 * (x - 0.5 * SV * nx) / W)
                                   - np.tanh(2 * (x - (1 - 0.5 * SV) * nx) / W))


def droplet(rhoi_V, rhoi_L, nx, ny, R, W=4.0):
    """Eq. (13): a liquid disc of radius R centred at (nx/2, ny/2)."""
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    d = np.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2) - R
    rv = np.asarray(rhoi_V, float)[:, None, None]
    rl = np.asarray(rhoi_L, float)[:, None, None]
    return 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2 * d / W)


def spinodal_point(P: OracleProblem, z, npts=400, B_max=0.6):
    """Total molar density on the fixed-z line, with b_m rho~ <= B_max, where
    the smallest stability eigenvalue is most negative (None if that part of
    the line never enters the spinodal).  B_max keeps the uniform state away
    from the nearly incompressible liquid branch, whose sound speed the
    lattice cannot carry."""
    z = np.asarray(z, float)
    bm = float(z @ P.b)
    rhos = np.linspace(0.02, B_max, npts) / bm
    lam = np.array([min_stability_eigenvalue(P, z * r) for r in rhos])
    k = int(np.argmin(lam))
    if lam[k] >= 0:
        return None
    return float(rhos[k]), float(lam[k])


def spinodal_temperature(make_problem, z, T_lo, T_hi, npts=160, tol=1e-6, B_max=0.6):
    """Highest temperature at which the fixed-z line (b_m rho~ <= B_max)
    enters the spinodal region (bisection on the sign of the most negative
    stability eigenvalue).  ``make_problem(T)`` returns an OracleProblem at T."""
    def deepest(T):
        P = make_problem(T)
        bm = float(np.asarray(z) @ P.b)
        rhos = np.linspace(0.02, B_max, npts) / bm
        return min(min_stability_eigenvalue(P, np.asarray(z) * r) for r in rhos)
    if deepest(T_lo) >= 0:
        return None
    lo, hi = T_lo, T_hi
    while deepest(hi) < 0:
        lo, hi = hi, 2 * hi
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if deepest(mid) < 0:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol * hi:
            break
    return lo
