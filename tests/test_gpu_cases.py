"""Cases 1-6 of Sec. 3.2 (flat-interface vapour-liquid equilibrium with one to
six n-alkanes) in physical units on the GPU.

Set-up as the paper states it: components C1..C6 of the component table,
equimolar z, T and the initial p of the case table; lattice units from R = 1,
a_C1 = 2/49, b_C1 = 2/21, M_C1 = 1 (physical molar masses relative to C1);
delta_ij = 0; tau = 1; kappa_ref = 0.02 on C1 (Eq. 6); a 400 x 2 periodic
D2Q9 lattice started from Eq. (15) at the flash of (T, p, z) with W = 4; 1e6
steps.  The test runs binary32 throughout (LBM_FP32): on 800 nodes the
binary64 path keeps eight SMs busy on the FP64 pipe and takes 1-3 minutes per
case; a binary64 run of all six cases gave the same densities and mole
fractions to the digits the paper prints.

Checks, at the phase centres (vapour x = 0, liquid x = nx/2):
* Cases 2-6: phase mass densities and mole fractions within 0.5 % (relative)
  of the oracle flash at the LBM's own pressure and conserved overall
  composition, which is the paper's comparison (its largest error is
  0.264909 %, Table IV).  Case 1: the Maxwell coexistence densities within
  5e-4 (the even/odd mode of the chemical potential bounds a one-component
  flat interface at T_r = 0.93, see the oracle's flat-interface pin).
* The paper's own LBM results (Table III): phase densities within 0.3 %,
  mole fractions within 5e-4 absolute (the paper prints four digits, and
  leaves R unstated: 8.314462618 is the reading, worth 1.5e-4 in the Case 1
  densities).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle.thermo import LatticeUnits, flash, maxwell
from oracle.workloads import slab

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NAMES = ["C1", "C2", "C3", "C4", "C5", "C6"]
NX, NY = 400, 2
STEPS = 1000000
PRECISION = 2  # LBM_FP32


def load_components():
    rows = {}
    for line in open(f"{GOLDEN}/components.txt"):
        if line.startswith("#") or not line.strip():
            continue
        name, pc, Tc, om, M = line.split()
        rows[name] = (float(pc), float(Tc), float(om), float(M))
    return rows


def load_vle():
    out = []
    for line in open(f"{GOLDEN}/vle_cases.txt"):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        xs = [float(v) for v in f[5:] if v != "-"]
        out.append((int(f[0]), float(f[1]), float(f[2]), f[3], float(f[4]), np.array(xs)))
    return out


def case_units(case):
    comp = load_components()
    rows = [r for r in load_vle() if r[0] == case]
    sel = [comp[n] for n in NAMES[:case]]
    lu = LatticeUnits([s[1] for s in sel], [s[0] for s in sel], [s[2] for s in sel], [s[3] for s in sel])
    return lu, rows


def run_case(case, steps=STEPS, precision=PRECISION):
    from paper_2306_10652_gb300 import lbmfug
    lu, rows = case_units(case)
    T, p0 = rows[0][1], rows[0][2]
    P = lu.problem(T)
    z = np.ones(case) / case
    if case == 1:
        _, rV, rL = maxwell(P)
        rhoi_V, rhoi_L, SV = np.array([rV]), np.array([rL]), 0.5
    else:
        fl = flash(P, lu.p(p0), z)
        assert fl is not None
        rhoi_V, rhoi_L, SV = fl.rhoi_V, fl.rhoi_L, fl.S_V
    rho_molar = np.repeat(slab(rhoi_V, rhoi_L, NX, SV)[:, None, None, :], NY, axis=2)  # [nc][1][ny][nx]
    rho_mass = rho_molar * lu.M[:, None, None, None]
    with lbmfug.Problem(0, NX, NY, 1, lu.a, lu.b, lu.omega, None, lu.T(T), 1.0, M=lu.M, kappa_ref=0.02,
                        precision=precision) as gp:
        gp.init_fields(rho_mass)
        gp.step(steps)
        mo = gp.moments(("rho", "p"))
    rm = mo["rho"][:, 0, 0, :] / lu.M[:, None]  # molar densities along x
    pr = mo["p"][0, 0, :]
    tot = rm.sum(axis=1)
    return {"case": case, "lu": lu, "P": P, "T": T, "rows": rows, "V": rm[:, 0], "L": rm[:, NX // 2],
            "p": 0.5 * (pr[0] + pr[NX // 2]), "z": tot / tot.sum()}


@pytest.fixture(scope="module")
def cases():
    return {c: run_case(c) for c in range(1, 7)}


def rel(a, b):
    return np.abs(np.asarray(a) / np.asarray(b) - 1.0)


def flash_errors(r):
    """Relative errors of the LBM phases against the flash at the LBM's own
    pressure and overall composition (Maxwell for one component):
    {phase: (density error, mole-fraction errors)}."""
    lu, P = r["lu"], r["P"]
    if r["case"] == 1:
        _, rV, rL = maxwell(P)
        return {"V": (float(rel(r["V"][0], rV)), np.zeros(1)), "L": (float(rel(r["L"][0], rL)), np.zeros(1))}
    fl = flash(P, r["p"], r["z"])
    assert fl is not None
    out = {}
    for ph, lbm, th, x_th in (("V", r["V"], fl.rhoi_V, fl.y), ("L", r["L"], fl.rhoi_L, fl.x)):
        out[ph] = (float(rel(lu.mass_density_kg_m3(lbm), lu.mass_density_kg_m3(th))), rel(lbm / lbm.sum(), x_th))
    return out


@pytest.mark.parametrize("case", range(1, 7))
def test_case_matches_flash_at_lbm_pressure(cases, case):
    tol = 5e-4 if case == 1 else 5e-3
    for ph, (e_rho, e_x) in flash_errors(cases[case]).items():
        assert e_rho <= tol and e_x.max() <= tol, (case, ph, e_rho, e_x)


@pytest.mark.parametrize("case", range(1, 7))
def test_case_matches_paper_table(cases, case):
    r = cases[case]
    lu = r["lu"]
    for (_, _, _, ph, rho_kg, xs) in r["rows"]:
        lbm = r["V"] if ph == "V" else r["L"]
        assert rel(lu.mass_density_kg_m3(lbm), rho_kg) <= 3e-3, (case, ph, lu.mass_density_kg_m3(lbm), rho_kg)
        assert np.abs(lbm / lbm.sum() - xs).max() <= 5e-4, (case, ph, lbm / lbm.sum(), xs)
