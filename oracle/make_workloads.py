"""Write the stored physical set-up of the synthetic workloads.

TEST INFRASTRUCTURE (calls only ``oracle/`` and the seeded generators).
Output: ``paper_2306_10652_gb300/workloads/spinodal_2048.json`` -- for
Nc = 1..10 the seeded PR parameters of the 2048 x 2048 spinodal-decomposition
workload (Sec. 3.5 analogue), the temperature and the uniform molar density
inside the spinodal region that the oracle's stability test selects.

Recipe (seed 2): a_i = 2/49 U[0.3, 3], b_i = 2/21 U[0.6, 2.0],
omega_i ~ U[0, 0.5], delta_ij ~ U[0, 0.15], z ~ Dirichlet(1..1).
T = 0.98 T*, where T* is the highest temperature at which the fixed-z line
(restricted to b_m rho~ <= 0.35) enters the spinodal region; rho~ = argmin
over that line of the smallest eigenvalue of
diag(rho~)^(1/2) d ln f/d rho~ diag(rho~)^(1/2).  Deeper quenches (0.95 T*)
or denser states made the seeded runs fail within 3000 steps at tau = 1,
kappa_ref = 0.02 (density ratios and sound speeds beyond what the lattice
carries); 0.98 T* with b_m rho~ <= 0.35 ran 3000 steps for every Nc.

Run:  python -m oracle.make_workloads
"""
from __future__ import annotations

import json
import os

import numpy as np

from paper_2306_10652_gb300 import synth

from .orc import OracleProblem
from .workloads import spinodal_point, spinodal_temperature

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "paper_2306_10652_gb300", "workloads", "spinodal_2048.json")
SEED = 2
T_FACTOR = 0.98
B_MAX = 0.35


def spinodal_case(nc: int):
    c = synth.pr_components(SEED, nc, a_range=(0.3, 3.0), b_range=(0.6, 2.0),
                            k_range=(0.0, 0.15))
    z = synth.dirichlet(SEED, nc)
    def make(T):
        return OracleProblem(0, 1, 1, 1, c["a"], c["b"], c["omega"], c["kij"], T=T)
    Tc = make(1.0).critical_temperatures()
    Tstar = spinodal_temperature(make, z, 0.3 * float(Tc.min()), float(Tc.max()), B_max=B_MAX)
    if Tstar is None:
        raise RuntimeError(f"Nc={nc}: no spinodal region on the fixed-z line")
    T = T_FACTOR * Tstar
    P = make(T)
    sp = spinodal_point(P, z, B_max=B_MAX)
    if sp is None:
        raise RuntimeError(f"Nc={nc}: the fixed-z line does not enter the spinodal region")
    rho, lam = sp
    return {"nc": nc, "a": c["a"].tolist(), "b": c["b"].tolist(), "omega": c["omega"].tolist(),
            "kij": c["kij"].tolist(), "z": z.tolist(), "T": T, "rho_molar_total": rho,
            "min_eigenvalue": lam, "T_star": Tstar, "tau": 1.0, "kappa_ref": 0.02}


def main():
    cases = [spinodal_case(nc) for nc in range(1, 11)]
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump({"workload": "spinodal decomposition, D2Q9 2048x2048 periodic",
                   "seed": SEED, "noise": "multiplicative 1 +- 0.01 U[-1,1], seed 2, stream 4",
                   "nx": 2048, "ny": 2048, "cases": cases}, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
