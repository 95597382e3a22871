"""The batched form (lbm_batch_*): many small problems in one persistent kernel.

* one step of each job against the oracle (binary32 bar: 1e-5 of max |g|);
* each job's result is bitwise the same alone, in a mix and at any CTA size;
* component mass of every job is conserved;
* jobs run to convergence reach the single-problem binary64 path's phase
  compositions within 1e-5 and the oracle flash within 1 %.
"""
from __future__ import annotations

import numpy as np
import pytest

from helpers import gpu_problem, oracle_problem, order_map, seeded_mixture, smooth_rho
from oracle.thermo import flash
from oracle.workloads import slab, two_phase_pressure
from paper_2306_10652_gb300 import synth

pytestmark = pytest.mark.gpu


def lb():
    from paper_2306_10652_gb300 import lbmfug
    return lbmfug


def job_set(seed, shapes, Tfacs, nc=3):
    c = seeded_mixture(seed, nc, 0, (1, 4, 64))
    Tc = oracle_problem(c, 0, (1, 1, 1)).critical_temperatures()
    jobs = []
    for k, ((ny, nx), tf) in enumerate(zip(shapes, Tfacs)):
        rho = smooth_rho(seed + k, c, (1, ny, nx), 0.02, 0.12)[:, 0]
        jobs.append((tf * Tc.mean(), rho))
    return c, jobs


SHAPES = [(4, 64), (3, 97), (4, 130), (2, 33), (5, 17), (1, 40)]
TFACS = [0.85, 0.9, 0.8, 0.95, 0.88, 0.92]


@pytest.mark.parametrize("precision", [2, 1])   # LBM_FP32, LBM_FP32DEV
def test_batch_one_step_matches_oracle(precision):
    c, jobs = job_set(5, SHAPES, TFACS)
    with lb().Batch(c["a"], c["b"], c["omega"], c["kij"], 1.0, jobs, precision=precision) as bt:
        bt.run(max_steps=1, check_every=1, tol=0.0)
        for k, (T, rho) in enumerate(jobs):
            ny, nx = rho.shape[1:]
            cc = dict(c, T=T)
            orc = oracle_problem(cc, 0, (1, ny, nx))
            ref = orc.moments(orc.step(orc.init_equilibrium(rho[:, None]), 1))["rho"][:, 0]
            got = bt.state(k)["rho"]
            assert np.abs(got / ref - 1).max() < 1e-5, k


def test_batch_alone_vs_mix_bitwise():
    c, jobs = job_set(7, SHAPES, TFACS)
    with lb().Batch(c["a"], c["b"], c["omega"], c["kij"], 1.0, jobs) as bt:
        bt.run(max_steps=300, check_every=100, tol=0.0)
        mix = [bt.state(k)["rho"] for k in range(len(jobs))]
    for k in (0, 3):
        for th in (128, 256, 512):
            with lb().Batch(c["a"], c["b"], c["omega"], c["kij"], 1.0, [jobs[k]]) as one:
                one.set_threads(th)
                one.run(max_steps=300, check_every=100, tol=0.0)
                assert np.array_equal(one.state(0)["rho"], mix[k]), (k, th)


def test_batch_mass_conserved():
    # above the mixture's critical region, so the smooth random states stay stable
    c, jobs = job_set(9, SHAPES, [1.05, 1.1, 1.15, 1.2, 1.1, 1.05])
    m0 = [rho.sum(axis=(1, 2)) for _, rho in jobs]
    with lb().Batch(c["a"], c["b"], c["omega"], c["kij"], 1.0, jobs) as bt:
        bt.run(max_steps=2000, check_every=500, tol=0.0)
        for k in range(len(jobs)):
            m = bt.state(k)["rho"].sum(axis=(1, 2))
            assert np.abs(m / m0[k] - 1).max() < 1e-9, k


def slab_jobs(seed, Tfacs, nx=64, ny=2, nc=3):
    c = seeded_mixture(seed, nc, 0, (1, ny, nx))
    Tc = oracle_problem(c, 0, (1, 1, 1)).critical_temperatures()
    jobs, cases = [], []
    for tf in Tfacs:
        cc = dict(c, T=tf * Tc.mean())
        orc = oracle_problem(cc, 0, (1, ny, nx))
        p, fl = two_phase_pressure(orc, np.ones(nc) / nc, 0.5)
        rho = np.repeat(slab(fl.rhoi_V, fl.rhoi_L, nx)[:, None, :], ny, axis=1)
        jobs.append((cc["T"], rho))
        cases.append((cc, orc))
    return c, jobs, cases


def test_batch_converges_to_binary64_and_flash():
    # seed 20 at 0.90 / 0.94 of the mean critical temperature: flat interfaces
    # that the binary64 path carries to equilibrium (several other seeded
    # ternaries at 0.86 - 0.9 diverge on every path: too large density ratios)
    c, jobs, cases = slab_jobs(20, [0.9, 0.94])
    with lb().Batch(c["a"], c["b"], c["omega"], c["kij"], 1.0, jobs) as bt:
        # binary32 storage: the state jitters at the binary32 resolution of the
        # populations, so "converged" is a density change below 2e-6 per 1000
        # steps (about 8 ulp of binary32 at the liquid densities here)
        nconv = bt.run(max_steps=200000, check_every=1000, tol=2e-6)
        diag = [(bt.state(k)["steps"], bt.state(k)["last_drho"]) for k in range(len(jobs))]
        assert nconv == len(jobs), diag
        for k, ((cc, orc), (T, rho0)) in enumerate(zip(cases, jobs)):
            st = bt.state(k)
            r = st["rho"][:, 0]
            nx = r.shape[1]
            xL, xV = r[:, nx // 2] / r[:, nx // 2].sum(), r[:, 0] / r[:, 0].sum()
            # the single-problem binary64 path to the same number of steps
            with gpu_problem(cc, 0, (1, 2, nx), precision=0) as gp:
                gp.init_fields(rho0[:, None])
                gp.step(st["steps"])
                m = gp.moments()
            r64 = m["rho"][:, 0, 0]
            assert np.abs(xL - r64[:, nx // 2] / r64[:, nx // 2].sum()).max() < 1e-5
            assert np.abs(xV - r64[:, 0] / r64[:, 0].sum()).max() < 1e-5
            # the flash at the LBM's own pressure and overall composition
            pm = 0.5 * (m["p"][0, 0, nx // 2] + m["p"][0, 0, 0])
            f2 = flash(orc, pm, r.sum(axis=1) / r.sum())
            # near the critical temperature the LBM-vs-flash deviation grows; the
            # paper's largest is 0.511047 % (Table VIII): allow 1 %
            assert np.abs(xL / f2.x - 1).max() < 1e-2 and np.abs(xV / f2.y - 1).max() < 1e-2
