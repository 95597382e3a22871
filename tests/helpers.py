"""Shared test helpers: paired oracle / CUDA problems on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import OracleProblem, lattice_info
from paper_2306_10652_gb300 import synth


def seeded_mixture(seed, nc, lattice=0, shape=(1, 8, 8), Tfac=0.85, **synth_kw):
    """Seeded PR parameters and a temperature Tfac * mean Tc (lattice units)."""
    c = synth.pr_components(seed, nc, **synth_kw)
    P0 = OracleProblem(lattice, shape[2], shape[1], shape[0], c["a"], c["b"], c["omega"], c["kij"], T=1.0)
    c["T"] = Tfac * float(P0.critical_temperatures().mean())
    return c


def oracle_problem(c, lattice, shape, tau=1.0, M=None, kappa_ref=0.02):
    return OracleProblem(lattice, shape[2], shape[1], shape[0], c["a"], c["b"], c["omega"], c["kij"],
                         T=c["T"], tau=tau, M=M, kappa_ref=kappa_ref)


def gpu_problem(c, lattice, shape, tau=1.0, M=None, kappa_ref=0.02, **opts):
    from paper_2306_10652_gb300 import lbmfug
    return lbmfug.Problem(lattice, shape[2], shape[1], shape[0], c["a"], c["b"], c["omega"],
                          c["kij"], c["T"], tau, M=M, kappa_ref=kappa_ref, **opts)


def order_map(lattice, gpu_e):
    """Index list to_orc with g_gpu[:, to_orc] in the oracle's velocity order."""
    _, _, e_orc, _ = lattice_info(lattice)
    return [int(np.where((gpu_e == v).all(axis=1))[0][0]) for v in e_orc]


def smooth_rho(seed, c, shape, lo=0.05, hi=0.6):
    """Random smooth molar-ish densities with b-scaled magnitude (B from lo to hi overall)."""
    nc = len(c["a"])
    return synth.random_state(seed, nc, shape, lo, hi) / np.asarray(c["b"])[:, None, None, None] / nc
