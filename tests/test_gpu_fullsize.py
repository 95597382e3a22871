"""Oracle parity at full size, in the launch configuration the benchmark
times: the spinodal workload (D2Q9 2048 x 2048, Nc = 10, seeded PR mixture,
+-1 % noise), one step, checked on sampled nodes; and a 5248 x 5248, Nc = 10
problem whose 8 Nc N population index passes 2^31, so the kernel with 64-bit
indexing runs.

One step at a node reads only nodes within distance 3 (the push of the
collided neighbours at distance 1, their force from mu at distance 2, mu
from psi at distance 3), so the oracle runs a periodic 9 x 9 patch of the
initial densities centred on the sample and its centre equals the full
problem's node.  The samples include the first and last rows of CTA
segments, the first and last columns of strips and the periodic corners.
Tolerances as in the one-step tests: populations within 2e-6 (binary32
storage, df64 thermodynamics) or 1e-5 (binary32 thermodynamics) of max
|g_i|; densities after the step within 2e-6 of max rho_i.
"""
from __future__ import annotations

import numpy as np
import pytest

from bench import initial_density, load_case
from helpers import order_map
from oracle import OracleProblem
from paper_2306_10652_gb300 import synth

pytestmark = pytest.mark.gpu

FP32DEV, FP32 = 1, 2
TOL = {FP32DEV: 2e-6, FP32: 1e-5}


def problem(case, nx, ny, precision):
    from paper_2306_10652_gb300 import lbmfug
    return lbmfug.Problem(0, nx, ny, 1, case["a"], case["b"], case["omega"], np.asarray(case["kij"]),
                          case["T"], case["tau"], precision=precision, kappa_ref=case["kappa_ref"],
                          monitor_every=1)


def samples(info, nx, ny, n_random, seed):
    ys = {0, ny - 1}
    for s in range(1, min(info["segs"], 6)):
        ys |= {s * info["seg_h"] - 1, s * info["seg_h"]}
    xs = {0, nx - 1}
    for k in range(1, min(info["nstrips"], 6)):
        xs |= {k * info["strip"] - 1, k * info["strip"]}
    pts = [(y, x) for y in sorted(ys)[:6] for x in sorted(xs)[:6]]
    rng = np.random.default_rng(seed)
    pts += [(int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(n_random)]
    return pts


def patch(field, y, x, r=4):
    ny, nx = field.shape[-2:]
    yy = np.arange(y - r, y + r + 1) % ny
    xx = np.arange(x - r, x + r + 1) % nx
    return np.ascontiguousarray(field[..., yy[:, None], xx[None, :]])


def oracle_center(case, rho_patch, M=None):
    nc = rho_patch.shape[0]
    orc = OracleProblem(0, 9, 9, 1, case["a"], case["b"], case["omega"], np.asarray(case["kij"]),
                        T=case["T"], tau=case["tau"], kappa_ref=case["kappa_ref"], M=M)
    g = orc.step(orc.init_equilibrium(rho_patch.reshape(nc, 1, 9, 9)), 1)
    return g[:, :, 0, 4, 4], orc.moments(g)["rho"][:, 0, 4, 4]


@pytest.mark.parametrize("precision", [FP32DEV, FP32], ids=["fp32dev", "fp32"])
def test_bench_workload_one_step_sampled(precision):
    d, case = load_case(10)
    nx, ny = d["nx"], d["ny"]
    rho = initial_density(d, case, nx, ny)
    with problem(case, nx, ny, precision) as gp:
        gp.init_fields(rho)
        info = gp.schedule_info()
        assert info["fused"] == 1 and info["seg_h"] >= 8, info
        rho0 = gp.moments(("rho",))["rho"][:, 0]          # the densities the state holds
        gp.step(1)
        g = gp.get_state()[:, order_map(0, gp.e), 0]        # [nc, 9, ny, nx]
    scale = np.abs(g).max(axis=(1, 2, 3))
    worst = 0.0
    for (y, x) in samples(info, nx, ny, 24, 7):
        ref, _ = oracle_center(case, patch(rho0, y, x))
        err = (np.abs(g[:, :, y, x] - ref).max(axis=1) / scale).max()
        worst = max(worst, err)
        assert err < TOL[precision], ((y, x), err)
    print(f"full-size one-step worst relative error {worst:.3e}")


@pytest.mark.parametrize("precision", [FP32DEV, FP32], ids=["fp32dev", "fp32"])
def test_64bit_index_kernel_sampled(precision):
    d, case = load_case(10)
    nx = ny = 5248
    assert 8 * 10 * nx * ny >= 2 ** 31
    z = np.asarray(case["z"])
    rho = (z[:, None, None] * case["rho_molar_total"]) * synth.multiplicative_noise(11, (10, ny, nx), 0.01)
    with problem(case, nx, ny, precision) as gp:
        gp.init_fields(rho[:, None])
        del rho
        info = gp.schedule_info()
        rho0 = gp.moments(("rho",))["rho"][:, 0]
        gp.step(1)
        rho1 = gp.moments(("rho",))["rho"][:, 0]
    scale = rho1.max(axis=(1, 2))
    for (y, x) in samples(info, nx, ny, 16, 8):
        _, ref = oracle_center(case, patch(rho0, y, x))
        err = (np.abs(rho1[:, y, x] - ref) / scale).max()
        assert err < 2e-6, ((y, x), err)
