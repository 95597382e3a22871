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

Also ``workloads/ternary_sweep.json``: the batched ternary-diagram sweep
(Sec. 3.3 analogue) -- 1024 flat-interface D2Q9 slabs, Nc = 3, shared PR
parameters (seed 20 of the flat-interface recipe: a_i = 2/49 U[0.6, 1.6],
b_i = 2/21 U[0.8, 1.2], delta_ij ~ U[0, 0.1]), ny = 4 and nx drawn from
{64, 96, ..., 512}, at four temperatures (0.88, 0.91, 0.94, 0.97) x the mean
Tc, 256 overall compositions each on a triangle grid (seed 3) and a vapour
volume fraction S_V ~ U[0.3, 0.7]; p is set by the flash to that S_V and the
slab starts from Eq. (15) at the flash phase densities.  Points with no
two-phase split, or with a liquid/vapour molar density ratio above 10 (the
LBM at tau = 1, kappa_ref = 0.02 diverged on such slabs), are redrawn from
the same stream.

And ``workloads/served_requests.json``: 24 served requests (seed 4), each
with its own Nc ~ U{2..10}, seeded PR parameters, T ~ U[0.88, 0.94] x mean
Tc, equimolar z, S_V ~ U[0.35, 0.65] and the flash phase densities, as a
D2Q9 slab (nx 64..256, ny 4..64), a D2Q9 droplet (64^2..128^2) or a D3Q19
slab box (24^3..48^3); Poisson arrival gaps with mean 0.05 s.  Each draw is
screened by a 20000-step oracle run of a two-node-thick slab of its own
state on its lattice and nx (tau = 1, kappa_ref = 0.02); draws that diverge
there are redrawn (several with liquid/vapour ratios of only 2 - 2.5 did).  Sizes are
scaled down from 64^2..1024^2 / 64^3..192^3 so that a bench run finishes in
minutes.

Run:  python -m oracle.make_workloads            (spinodal)
      python -m oracle.make_workloads ternary    (batched sweep)
      python -m oracle.make_workloads serve      (served requests)
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


TERNARY_SEED = 3
TERNARY_PARAM_SEED = 20
TERNARY_T = (0.88, 0.91, 0.94, 0.97)


def _ternary_point(args):
    """Flash of one sweep point (runs in a worker process)."""
    T, z, SV = args
    from .thermo import flash as _flash  # noqa: F401
    from .workloads import two_phase_pressure
    c = synth.pr_components(TERNARY_PARAM_SEED, 3)
    P = OracleProblem(0, 1, 1, 1, c["a"], c["b"], c["omega"], c["kij"], T=T)
    res = two_phase_pressure(P, np.asarray(z), SV, tol=1e-9, npts=80)
    if res is None:
        return None
    p, fl = res
    if fl.rho_L * float(fl.x @ np.ones(3)) / (fl.rho_V * float(fl.y @ np.ones(3))) > 10.0:
        return None  # density ratio beyond what tau = 1 carries: redrawn
    return {"T": T, "z": list(z), "S_V": SV, "p": p, "rhoi_V": fl.rhoi_V.tolist(),
            "rhoi_L": fl.rhoi_L.tolist(), "x": fl.x.tolist(), "y": fl.y.tolist()}


def ternary_sweep(njobs=1024, procs=8):
    import multiprocessing as mp
    c = synth.pr_components(TERNARY_PARAM_SEED, 3)
    Tc = OracleProblem(0, 1, 1, 1, c["a"], c["b"], c["omega"], c["kij"], T=1.0).critical_temperatures()
    rng = synth.rng_for(TERNARY_SEED, 7)
    per_T = njobs // len(TERNARY_T)
    jobs = []
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for tf in TERNARY_T:
            T = tf * float(Tc.mean())
            got = []
            while len(got) < per_T:
                need = per_T - len(got)
                cand = []
                for _ in range(2 * need):
                    # a point of the triangle grid of step 1/32, away from the edges
                    i, j = rng.integers(1, 31, 2)
                    if i + j >= 32:
                        i, j = 32 - i, 32 - j
                    z = np.array([i, j, 32 - i - j], float) / 32.0
                    cand.append((T, tuple(z), float(rng.uniform(0.3, 0.7))))
                for r in pool.map(_ternary_point, cand):
                    if r is not None and len(got) < per_T:
                        got.append(r)
            jobs += got
    nxs = [int(v) for v in rng.choice(np.arange(64, 513, 32), size=len(jobs))]
    for jb, nx in zip(jobs, nxs):
        jb["nx"], jb["ny"] = nx, 4
    return {"workload": "batched ternary-diagram sweep, 1024 D2Q9 flat-interface slabs, Nc=3",
            "seed": TERNARY_SEED, "param_seed": TERNARY_PARAM_SEED, "a": c["a"].tolist(),
            "b": c["b"].tolist(), "omega": c["omega"].tolist(), "kij": c["kij"].tolist(),
            "tau": 1.0, "kappa_ref": 0.02, "W": 4.0, "jobs": jobs}


SERVE_SEED = 4


def _serve_request(k):
    """One request of the served workload (runs in a worker process)."""
    from .workloads import two_phase_pressure
    rng = synth.rng_for(SERVE_SEED, 100 + k)
    for attempt in range(40):
        nc = int(rng.integers(2, 11))
        c = synth.pr_components(SERVE_SEED * 1000 + 37 * k + attempt, nc)
        P = OracleProblem(0, 1, 1, 1, c["a"], c["b"], c["omega"], c["kij"], T=1.0)
        T = float(rng.uniform(0.88, 0.94)) * float(P.critical_temperatures().mean())
        P = OracleProblem(0, 1, 1, 1, c["a"], c["b"], c["omega"], c["kij"], T=T)
        SV = float(rng.uniform(0.35, 0.65))
        res = two_phase_pressure(P, np.ones(nc) / nc, SV, tol=1e-9, npts=80)
        if res is None:
            continue
        p, fl = res
        if fl.rho_L / fl.rho_V > 10.0:
            continue
        kind = str(rng.choice(["slab", "droplet", "box"], p=[0.45, 0.35, 0.2]))
        if kind == "slab":
            geo = {"lattice": 0, "nx": int(rng.choice([64, 96, 128, 192, 256])), "ny": int(rng.choice([4, 16, 64])), "nz": 1}
        elif kind == "droplet":
            n = int(rng.choice([64, 96, 128]))
            geo = {"lattice": 0, "nx": n, "ny": n, "nz": 1}
        else:
            n = int(rng.choice([24, 32, 48]))
            geo = {"lattice": 1, "nx": n, "ny": n, "nz": n}
        if not _slab_survives(c, T, geo["lattice"], geo["nx"], SV, fl):
            continue  # diverges at tau = 1 on every path: redrawn
        return {"nc": nc, "a": c["a"].tolist(), "b": c["b"].tolist(), "omega": c["omega"].tolist(),
                "kij": c["kij"].tolist(), "T": T, "p": p, "S_V": SV, "kind": kind,
                "rhoi_V": fl.rhoi_V.tolist(), "rhoi_L": fl.rhoi_L.tolist(), **geo}
    return None


SERVE_SCREEN_STEPS = 20000


def _slab_survives(c, T, lattice, nx, SV, fl, steps=SERVE_SCREEN_STEPS):
    """Stability screen of one request: the oracle runs a flat Eq. (15) slab of
    the request's own mixture, temperature, phase densities, lattice and nx
    (two nodes thick) for ``steps`` steps at tau = 1, kappa_ref = 0.02.  Some
    splits with modest density ratios still diverge there (all paths, binary64
    included); a thin slab shows it at a small fraction of the cost of the
    full request."""
    from .workloads import slab
    nz = 2 if lattice == 1 else 1
    P = OracleProblem(lattice, nx, 2, nz, c["a"], c["b"], c["omega"], c["kij"], T=T)
    rho = np.broadcast_to(slab(fl.rhoi_V, fl.rhoi_L, nx, SV)[:, None, None, :],
                          (len(c["a"]), nz, 2, nx)).copy()
    g = P.init_equilibrium(rho)
    try:
        for _ in range(steps // 1000):
            g = P.step(g, 1000)
    except RuntimeError:  # non-finite densities
        return False
    return bool(np.isfinite(P.moments(g)["rho"]).all())


def served_requests(n=24, procs=8):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as pool:
        reqs = [r for r in pool.map(_serve_request, range(n)) if r is not None]
    rng = synth.rng_for(SERVE_SEED, 1)
    gaps = rng.exponential(0.05, len(reqs))
    for r, g in zip(reqs, gaps):
        r["arrival_gap_s"] = float(g)
    return {"workload": "served phase-equilibrium requests: D2Q9 slabs and droplets, D3Q19 slab boxes, Nc 2..10",
            "seed": SERVE_SEED, "arrival": "Poisson, mean gap 0.05 s", "tau": 1.0, "kappa_ref": 0.02, "W": 4.0,
            "requests": reqs}


def main():
    if len(__import__("sys").argv) > 1 and __import__("sys").argv[1] == "serve":
        out = os.path.join(os.path.dirname(OUT), "served_requests.json")
        with open(out, "w") as f:
            json.dump(served_requests(), f)
        print(out)
        return
    if len(__import__("sys").argv) > 1 and __import__("sys").argv[1] == "ternary":
        out = os.path.join(os.path.dirname(OUT), "ternary_sweep.json")
        with open(out, "w") as f:
            json.dump(ternary_sweep(), f)
        print(out)
        return
    cases = [spinodal_case(nc) for nc in range(1, 11)]
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump({"workload": "spinodal decomposition, D2Q9 2048x2048 periodic",
                   "seed": SEED, "noise": "multiplicative 1 +- 0.01 U[-1,1], seed 2, stream 4",
                   "nx": 2048, "ny": 2048, "cases": cases}, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
