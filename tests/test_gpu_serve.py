"""The served form (lbm_server_*): admission by a memory budget, overlapping
jobs, retirement of finished or failed jobs, identical results alone and in
the mix."""
from __future__ import annotations

import time

import numpy as np
import pytest

from helpers import gpu_problem, oracle_problem, seeded_mixture, smooth_rho
from oracle.thermo import maxwell
from oracle.workloads import slab
from paper_2306_10652_gb300 import synth

pytestmark = pytest.mark.gpu

FP32DEV, FP32 = 1, 2


def lb():
    from paper_2306_10652_gb300 import lbmfug
    return lbmfug


def requests():
    """Mixed jobs: D2Q9 slabs and a random field, a D3Q19 box."""
    out = []
    for k, (lat, shape, nc) in enumerate([(0, (1, 4, 96), 2), (0, (1, 24, 40), 3), (1, (8, 10, 12), 2),
                                          (0, (1, 6, 130), 4)]):
        c = seeded_mixture(100 + k, nc, lat, shape)
        rho = smooth_rho(100 + k, c, shape, 0.02, 0.12)
        out.append((lat, c, rho))
    return out


def run_alone(lat, c, rho, steps, precision):
    with gpu_problem(c, lat, rho.shape[1:], precision=precision) as gp:
        gp.init_fields(rho)
        gp.step(steps)
        return gp.moments(("rho",))["rho"]


@pytest.mark.parametrize("precision", [FP32DEV, FP32])
def test_results_alone_equal_mix(precision):
    reqs = requests()
    with lb().Server(0.8, max_active=8) as srv:
        ids = [srv.submit(lat, c["a"], c["b"], c["omega"], c["kij"], c["T"], 1.0, rho, precision=precision,
                          check_every=250, max_steps=1000, tol=0.0) for lat, c, rho in reqs]
        srv.wait_all()
        for jid, (lat, c, rho) in zip(ids, reqs):
            p = srv.poll(jid)
            assert p["state"] == "exhausted" and p["steps"] == 1000 and p["latency_s"] > 0
            assert np.array_equal(srv.result(jid), run_alone(lat, c, rho, 1000, precision))
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["peak_bytes"] <= st["budget_bytes"]


def test_admission_respects_budget():
    lbmfug = lb()
    reqs = requests()[:3]
    import torch
    total = torch.cuda.get_device_properties(0).total_memory
    need = max(lbmfug.lbm_server_estimate_bytes(lat, rho.shape[3], rho.shape[2], rho.shape[1], rho.shape[0],
                                                FP32DEV) for lat, c, rho in reqs)
    frac = 1.5 * need / total          # room for one job at a time
    with lbmfug.Server(frac, max_active=8) as srv:
        ids = [srv.submit(lat, c["a"], c["b"], c["omega"], c["kij"], c["T"], 1.0, rho, precision=FP32DEV,
                          check_every=200, max_steps=400, tol=0.0) for lat, c, rho in reqs]
        srv.wait_all()
        st = srv.stats()
        assert st["peak_bytes"] <= st["budget_bytes"] < 2 * need
        assert all(srv.poll(j)["state"] == "exhausted" for j in ids)
        # one job at a time: the two later requests waited for memory with slots free
        adm = srv.admission()
        assert adm["peak_active"] == 1 and adm["memory_waits"] == 2, adm
        times = [srv.times(j) for j in ids]
        assert all(q >= 0.0 and r > 0.0 for q, r in times)
        assert times[2][0] >= times[0][1]  # the third queued at least as long as the first ran
        # a request that can never fit is refused at submission
        lat, c, rho = reqs[0]
        big = np.ones((2, 1, 512, 1024)) * 0.1
        with pytest.raises(lbmfug.LbmError) as e:
            srv.submit(0, c["a"], c["b"], c["omega"], c["kij"], c["T"], 1.0, big, precision=FP32DEV)
        assert e.value.status == lbmfug.LBM_ENOMEM


def test_failed_job_is_retired_and_others_finish():
    # a pure fluid far below its critical temperature (liquid/vapour ratio ~44)
    # diverges at tau = 1: its densities become non-finite
    cc = synth.pr_components(9, 1)
    orc = oracle_problem(dict(a=cc["a"], b=cc["b"], omega=cc["omega"], kij=None, T=1.0), 0, (1, 1, 64))
    T = 0.8 * orc.critical_temperatures()[0]
    orc = oracle_problem(dict(a=cc["a"], b=cc["b"], omega=cc["omega"], kij=None, T=T), 0, (1, 1, 64))
    psat, rV, rL = maxwell(orc)
    bad = np.repeat(slab(np.array([rV]), np.array([rL]), 64)[:, None, None, :], 2, axis=2)
    reqs = requests()[:2]
    with lb().Server(0.8, max_active=4) as srv:
        jb = srv.submit(0, cc["a"], cc["b"], cc["omega"], None, T, 1.0, bad, precision=FP32DEV,
                        check_every=1000, max_steps=40000, tol=0.0)
        ids = [srv.submit(lat, c["a"], c["b"], c["omega"], c["kij"], c["T"], 1.0, rho, precision=FP32DEV,
                          check_every=1000, max_steps=3000, tol=0.0) for lat, c, rho in reqs]
        srv.wait_all()
        pb = srv.poll(jb)
        assert pb["state"] == "failed" and pb["status"] != 0
        assert all(srv.poll(j)["state"] == "exhausted" for j in ids)


@pytest.mark.parametrize("lat,shape,nc,precision", [
    (0, (1, 512, 640), 10, FP32DEV), (0, (1, 256, 384), 4, 0), (1, (48, 56, 64), 7, FP32DEV),
    (1, (32, 40, 48), 3, 0)])
def test_estimate_covers_allocation(lat, shape, nc, precision):
    """lbm_server_estimate_bytes is at least what a handle of that size
    allocates on the device (measured as the drop of free device memory
    across initialisation), and not far above it."""
    import torch
    lbmfug = lb()
    c = seeded_mixture(140, nc, lat, shape)
    rho = smooth_rho(140, c, shape, 0.02, 0.12)
    est = lbmfug.lbm_server_estimate_bytes(lat, shape[2], shape[1], shape[0], nc, precision)
    small = (1, 8, 16) if lat == 0 else (4, 5, 6)  # loads the kernels before the measurement
    with gpu_problem(seeded_mixture(141, nc, lat, small), lat, small, precision=precision) as gp:
        gp.init_fields(smooth_rho(141, seeded_mixture(141, nc, lat, small), small, 0.02, 0.12))
        gp.step(2)
        gp.convergence()
        gp.synchronize()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    with gpu_problem(c, lat, shape, precision=precision) as gp:
        gp.init_fields(rho)
        gp.step(2)
        gp.convergence()  # allocates the convergence snapshot
        gp.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    assert used <= est, (used, est)
    assert est <= 1.3 * used + (64 << 20), (used, est)
