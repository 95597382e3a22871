"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances:
* binary64 storage, one step: max |g_gpu - g_orc| <= 1e-12 * max |g_i| per
  component.  The two sides differ only in the order of roundings: a few
  hundred binary64 operations per node-step at 1.1e-16 each, with the
  gradient differences amplifying relative errors of ln f by at most the
  ratio |ln f| / |grad ln f| (about 10 on these smooth fields).
* binary64, 1000 steps of the flat-interface case: |rho_gpu - rho_orc| <= 1e-9
  (rounding differences of 1e-15 per step, growing at most linearly on a
  stable interface: 1e-12 per 1000 steps, with three orders of margin for
  the slow modes of the interface).
* binary32 deviation storage, one step: within 2e-6 of max |g_i|.  A stored
  moving population is rounded once to binary32 (2^-24 = 6e-8 of its size)
  and the collision adds a few binary32 roundings of terms as large as
  rho_i / 9; 2e-6 of max |g_i| (dominated by the rest population) covers
  them with a factor of about 5.
* binary32 thermodynamics (LBM_FP32), one step: within 1e-5, since ln f_i
  from the hardware logarithm (absolute error 2^-21.4) enters the force
  through differences scaled by RT / |grad|.
* component mass within 1e-6 relative (the density pairs are exact to
  2^-48; the 1e-6 is the bar of the configuration), converged phase mole
  fractions within 1e-5 of the binary64 path (the bar of the configuration).
"""
from __future__ import annotations

import numpy as np
import pytest

from helpers import gpu_problem, oracle_problem, order_map, seeded_mixture, smooth_rho
from oracle.thermo import flash
from oracle.workloads import slab, two_phase_pressure
from paper_2306_10652_gb300 import synth

pytestmark = pytest.mark.gpu

FP64, FP32DEV, FP32 = 0, 1, 2
THREEPASS, AUTO, FUSED, MULTIPASS = 1, 0, 2, 3


def lb():
    from paper_2306_10652_gb300 import lbmfug
    return lbmfug


def one_step_case(seed, nc, lattice, shape, tau=1.0, Mrand=False, precision=FP64, schedule=THREEPASS,
                  nsteps=1, Tfac=0.85, lo=0.02, hi=0.12):
    c = seeded_mixture(seed, nc, lattice, shape, Tfac=Tfac)
    M = synth.uniform(seed, 0.5, 2.0, nc) if Mrand else None
    orc = oracle_problem(c, lattice, shape, tau=tau, M=M)
    rho = smooth_rho(seed, c, shape, lo, hi) * (1.0 if M is None else M[:, None, None, None])
    u = synth.random_velocity(seed, orc.D, shape, 1e-3)
    g0 = orc.init_equilibrium(rho, u)
    g_ref = orc.step(g0, nsteps)
    with gpu_problem(c, lattice, shape, tau=tau, M=M, precision=precision, schedule=schedule) as gp:
        gp.init_fields(rho, u)
        gp.step(nsteps)
        g = gp.get_state()[:, order_map(lattice, gp.e)]
    scale = np.abs(g_ref).max(axis=(1, 2, 3, 4), keepdims=True)
    return float((np.abs(g - g_ref) / scale).max())


CASES = [
    # seed, nc, lattice, shape (nz, ny, nx), tau, random M
    (0, 1, 0, (1, 8, 8), 1.0, False),
    (1, 2, 0, (1, 7, 13), 0.8, True),
    (2, 3, 0, (1, 33, 70), 1.0, False),
    (3, 5, 0, (1, 5, 131), 1.3, True),
    (4, 10, 0, (1, 16, 20), 1.0, False),
    (5, 16, 0, (1, 6, 9), 1.0, True),
    (6, 2, 0, (1, 1, 9), 1.0, False),
    (7, 2, 0, (1, 4, 1), 1.0, False),
    (8, 2, 1, (5, 6, 7), 1.0, True),
    (9, 3, 1, (4, 4, 4), 0.9, False),
    (10, 10, 1, (3, 5, 6), 1.0, False),
]


@pytest.mark.parametrize("case", CASES, ids=[f"lat{c[2]}-nc{c[1]}-{c[3]}" for c in CASES])
@pytest.mark.parametrize("schedule", [THREEPASS, AUTO])
def test_one_step_fp64(case, schedule):
    seed, nc, lattice, shape, tau, Mr = case
    assert one_step_case(seed, nc, lattice, shape, tau, Mr, FP64, schedule) < 1e-12


@pytest.mark.parametrize("case", CASES[:6] + CASES[8:11], ids=lambda c: f"lat{c[2]}-nc{c[1]}")
@pytest.mark.parametrize("schedule", [THREEPASS, AUTO, MULTIPASS])
def test_one_step_fp32dev(case, schedule):
    seed, nc, lattice, shape, tau, Mr = case
    assert one_step_case(seed, nc, lattice, shape, tau, Mr, FP32DEV, schedule) < 2e-6


@pytest.mark.parametrize("case", CASES[:6], ids=lambda c: f"lat{c[2]}-nc{c[1]}")
def test_one_step_fp32(case):
    """Binary32 thermodynamics (fused schedule): one step within 1e-5 of max |g_i|."""
    seed, nc, lattice, shape, tau, Mr = case
    assert one_step_case(seed, nc, lattice, shape, tau, Mr, FP32, AUTO) < 1e-5


STRIP_CASES = [
    # seed, nc, shape (nz, ny, nx), steps: ragged strips and segments, periodic wrap
    (90, 2, (1, 3, 300), 1),
    (91, 3, (1, 130, 127), 1),
    (92, 10, (1, 2, 253), 3),
    (93, 7, (1, 64, 5), 1),
    (94, 2, (1, 1, 1), 2),
    (95, 9, (1, 37, 250), 2),
    (96, 1, (1, 9, 250), 2),
    (97, 16, (1, 5, 131), 1),
]


@pytest.mark.parametrize("case", STRIP_CASES, ids=lambda c: f"nc{c[1]}-{c[2][1]}x{c[2][2]}")
def test_fp32_fused_strips(case):
    """Binary32 fused kernels (all components of a column in one thread for
    Nc = 1, split over two threads for Nc >= 2) against the oracle: within
    1e-5 of max |g_i| after one to three steps."""
    seed, nc, shape, steps = case
    assert one_step_case(seed, nc, 0, shape, precision=FP32, schedule=AUTO, nsteps=steps) < 1e-5


def test_ten_steps_fp64_two_phase():
    # liquid-range densities inside the two-phase region: strong forces
    assert one_step_case(11, 3, 0, (1, 24, 40), nsteps=10, lo=0.05, hi=0.6) < 1e-11


def flat_interface_case(seed=0, nx=128, ny=4, nc=2):
    """Binary slab, Eq. (15) at the flash densities for S_V = 0.5, with 1e-3
    multiplicative noise (the flat-interface workload)."""
    c = seeded_mixture(seed, nc, 0, (1, ny, nx))
    orc = oracle_problem(c, 0, (1, ny, nx))
    z = np.ones(nc) / nc
    p, fl = two_phase_pressure(orc, z, 0.5)
    prof = slab(fl.rhoi_V, fl.rhoi_L, nx)                       # [nc, nx]
    rho = np.repeat(prof[:, None, None, :], ny, axis=2)
    rho = rho * synth.multiplicative_noise(seed, rho.shape, 1e-3)
    return c, orc, rho


@pytest.mark.parametrize("schedule", [THREEPASS, AUTO])
def test_flat_interface_1000_steps_fp64(schedule):
    c, orc, rho = flat_interface_case()
    ref = orc.moments(orc.step(orc.init_equilibrium(rho), 1000))
    with gpu_problem(c, 0, orc.shape, precision=FP64, schedule=schedule) as gp:
        gp.init_fields(rho)
        gp.step(1000)
        m = gp.moments()
    assert np.abs(m["rho"] - ref["rho"]).max() <= 1e-9
    assert np.abs(m["u"] - ref["u"]).max() <= 1e-9
    assert np.abs(m["lnf"] - ref["lnf"]).max() <= 1e-8
    assert np.abs(m["p"] - ref["p"]).max() <= 1e-9


@pytest.mark.parametrize("nc", [2, 10])
@pytest.mark.parametrize("schedule,prec32", [(THREEPASS, FP32DEV), (AUTO, FP32DEV), (AUTO, FP32)])
def test_fp32dev_mass_and_equilibrium(schedule, prec32, nc):
    """Binary32 deviation storage against the binary64 path on a flat
    interface (binary and ten-component mixtures, seed 0): per-component
    mass within 1e-6 relative, and the converged phase mole fractions (phase
    centres, same sublattice) within 1e-5, after 4e4 steps."""
    c, orc, rho = flat_interface_case(nx=64, ny=2, nc=nc)
    m0 = orc.mass(orc.init_equilibrium(rho))
    res = {}
    for prec in (FP64, prec32):
        with gpu_problem(c, 0, orc.shape, precision=prec, schedule=schedule) as gp:
            gp.init_fields(rho)
            gp.step(1000)
            mass = gp.mass()
            if prec != FP64:
                assert np.abs(mass / m0 - 1).max() <= 1e-6
            gp.step(39000)
            r = gp.moments(("rho",))["rho"][:, 0, 0]
            res[prec] = (r[:, 32] / r[:, 32].sum(), r[:, 0] / r[:, 0].sum())
            if prec != FP64:
                assert np.abs(gp.mass() / m0 - 1).max() <= 1e-6
    for k in range(2):
        assert np.abs(res[prec32][k] - res[FP64][k]).max() <= 1e-5, (res[prec32][k], res[FP64][k])


@pytest.mark.parametrize("lattice,shape,nc", [(0, (1, 12, 17), 3), (1, (4, 5, 6), 2)])
def test_moments_match_oracle(lattice, shape, nc):
    c = seeded_mixture(21, nc, lattice, shape)
    orc = oracle_problem(c, lattice, shape)
    rho = smooth_rho(21, c, shape)
    u = synth.random_velocity(21, orc.D, shape, 1e-3)
    g = orc.step(orc.init_equilibrium(rho, u), 2)
    ref = orc.moments(g)
    with gpu_problem(c, lattice, shape) as gp:
        e_map = order_map(lattice, gp.e)
        inv = np.empty(len(e_map), int)
        inv[e_map] = np.arange(len(e_map))
        gp.set_state(g[:, inv])                 # oracle order -> library order
        m = gp.moments()
        assert np.allclose(gp.get_state()[:, e_map], g, rtol=0, atol=0)
    for k in ("rho", "u", "p", "lnf"):
        scale = max(np.abs(ref[k]).max(), 1e-30)
        assert np.abs(m[k] - ref[k]).max() <= 1e-13 * scale + 1e-15, k


@pytest.mark.parametrize("precision,schedule", [(FP64, THREEPASS), (FP64, AUTO), (FP32DEV, AUTO),
                                                (FP32, AUTO), (FP32DEV, MULTIPASS)])
def test_mass_conservation_and_uniform_fixed_point(precision, schedule):
    shape = (1, 40, 70)
    c = seeded_mixture(31, 3, 0, shape)
    rho = smooth_rho(31, c, shape)
    with gpu_problem(c, 0, shape, precision=precision, schedule=schedule) as gp:
        gp.init_fields(rho)
        m0 = gp.mass()
        gp.step(50)
        m1 = gp.mass()
        tol = 1e-13 if precision == FP64 else 1e-6
        assert np.abs(m1 / m0 - 1).max() < tol
    uni = np.ones((3,) + shape) * (0.3 / np.asarray(c["b"])[:, None, None, None] / 3)
    with gpu_problem(c, 0, shape, precision=precision, schedule=schedule) as gp:
        gp.init_fields(uni)
        g0 = gp.get_state()
        gp.step(5)
        assert np.array_equal(gp.get_state(), g0)


def test_convergence_monitor_and_nonfinite():
    shape = (1, 16, 16)
    c = seeded_mixture(41, 2, 0, shape)
    rho = smooth_rho(41, c, shape)
    with gpu_problem(c, 0, shape) as gp:
        gp.init_fields(rho)
        assert gp.convergence() == float("inf")
        gp.step(10)
        d1 = gp.convergence()
        assert 0 < d1 < 1
        assert gp.convergence() == 0.0     # no steps since the snapshot
        g = gp.get_state()
        g[0, 0, 0, 3, 3] = np.inf
        with pytest.raises(lb().LbmError):  # non-finite state is rejected on the host
            gp.set_state(g)


def test_device_buffers_and_stream():
    import torch
    shape = (1, 9, 14)
    c = seeded_mixture(51, 2, 0, shape)
    rho = smooth_rho(51, c, shape)
    s = torch.cuda.Stream()
    with gpu_problem(c, 0, shape, stream=s.cuda_stream) as gp:
        d_rho = torch.from_numpy(rho.copy()).cuda()
        gp.init_fields_device(d_rho.reshape(-1))
        gp.step(4)
        out = torch.empty_like(d_rho)
        gp.moments_device(d_rho=out)
        gp.synchronize()
        host = gp.moments(("rho",))["rho"]
    assert np.array_equal(out.cpu().numpy(), host)


def test_zero_steps_and_step_count():
    shape = (1, 5, 5)
    c = seeded_mixture(61, 1, 0, shape)
    rho = smooth_rho(61, c, shape)
    with gpu_problem(c, 0, shape) as gp:
        gp.init_fields(rho)
        g0 = gp.get_state()
        gp.step(0)
        assert np.array_equal(gp.get_state(), g0)
        gp.step(3)
        assert gp.step_count() == 3


@pytest.mark.parametrize("precision", [FP64, FP32DEV, FP32])
def test_monitor_matches_mass(precision):
    """The fused per-step mass monitor equals the separate reduction."""
    shape = (1, 37, 300)
    c = seeded_mixture(71, 3, 0, shape)
    rho = smooth_rho(71, c, shape)
    with gpu_problem(c, 0, shape, precision=precision, monitor_every=5) as gp:
        gp.init_fields(rho)
        gp.step(10)
        m, at, nf = gp.monitor()
        assert at == 10 and not nf
        ref = gp.mass()
        assert np.allclose(m, ref, rtol=1e-12 if precision == FP64 else 1e-6, atol=0)


def test_fused_matches_threepass_many_shapes():
    """Fused and three-pass schedules agree step by step (binary64) on shapes
    that exercise ragged strips and segments and periodic wrap."""
    for k, shape in enumerate([(1, 3, 300), (1, 130, 127), (1, 2, 253), (1, 64, 5), (1, 1, 1)]):
        c = seeded_mixture(80 + k, 2, 0, shape)
        rho = smooth_rho(80 + k, c, shape)
        out = []
        for sched in (THREEPASS, FUSED):
            with gpu_problem(c, 0, shape, precision=FP64, schedule=sched) as gp:
                gp.init_fields(rho, synth.random_velocity(k, 2, shape, 1e-3))
                gp.step(7)
                out.append(gp.get_state())
        scale = np.abs(out[0]).max()
        assert np.abs(out[0] - out[1]).max() <= 1e-12 * scale, shape


@pytest.mark.parametrize("lattice,shape,nc,steps", [(1, (6, 7, 9), 3, 5), (1, (5, 4, 6), 10, 3), (0, (1, 33, 70), 4, 5),
                                                   (1, (5, 9, 70), 4, 3), (1, (3, 5, 33), 7, 2)])
def test_multipass_several_steps(lattice, shape, nc, steps):
    """The multi-pass schedule (density update and psi of the next step in one
    pass) against the oracle over several steps: within 2e-6 of max |g_i|
    per step (a few binary32 roundings per step on each population).  The
    shapes include boxes whose rows are longer than one warp and ragged
    against the 256-node CTAs, and boxes smaller than one CTA."""
    err = one_step_case(300 + nc, nc, lattice, shape, precision=FP32DEV, schedule=MULTIPASS, nsteps=steps)
    assert err < 2e-6 * steps, err


def test_multipass_is_the_d3q19_default_for_fp32dev():
    """AUTO runs LBM_FP32DEV on D3Q19 with the multi-pass schedule: three
    launches per step (plus one psi pass after initialisation)."""
    shape = (6, 5, 4)
    c = seeded_mixture(310, 3, 1, shape)
    rho = smooth_rho(310, c, shape)
    with gpu_problem(c, 1, shape, precision=FP32DEV) as gp:
        gp.init_fields(rho)
        l0 = gp.launch_count()
        gp.step(4)
        assert gp.launch_count() - l0 == 1 + 3 * 4
        assert gp.schedule_info()["fused"] == 0


@pytest.mark.parametrize("precision", [FP64, FP32DEV, FP32], ids=["fp64", "fp32dev", "fp32"])
def test_launch_geometry_changes_no_result(precision):
    """The fused kernels' result does not depend on the launch geometry (each
    node's arithmetic and the order of its density sums are the same in every
    strip and segment): forced strip widths and segment heights, the tuned
    geometry and the built-in one give bitwise equal states."""
    shape = (1, 45, 200)
    c = seeded_mixture(320, 4, 0, shape)
    rho = smooth_rho(320, c, shape)
    u = synth.random_velocity(320, 2, shape, 1e-3)
    out = []
    for kw in (dict(tune=0), dict(tune=1), dict(strip=37, seg_h=5), dict(strip=100, seg_h=45),
               dict(strip=7, seg_h=1), dict(strip=61, seg_h=7)):
        with gpu_problem(c, 0, shape, precision=precision, schedule=FUSED, **kw) as gp:
            gp.init_fields(rho, u)
            gp.step(6)
            out.append(gp.get_state())
            info = gp.schedule_info()
            if "strip" in kw:
                assert (info["strip"], info["seg_h"]) == (kw["strip"], kw["seg_h"]), info
    for o in out[1:]:
        assert np.array_equal(o, out[0])


@pytest.mark.parametrize("precision,schedule,lattice,shape", [
    (FP32DEV, FUSED, 0, (1, 40, 130)), (FP32, FUSED, 0, (1, 40, 130)), (FP64, FUSED, 0, (1, 12, 30)),
    (FP32DEV, MULTIPASS, 1, (6, 7, 9)), (FP64, THREEPASS, 1, (4, 5, 6))],
    ids=["fp32dev-fused", "fp32-fused", "fp64-fused", "fp32dev-multipass-d3q19", "fp64-threepass-d3q19"])
def test_step_graph_equals_step(precision, schedule, lattice, shape):
    """lbm_step_graph (the steps captured once into a CUDA graph per starting
    buffer and replayed) gives bitwise the states of lbm_step, for odd and
    even step counts and repeated replays."""
    c = seeded_mixture(330, 3, lattice, shape)
    rho = smooth_rho(330, c, shape)
    out = []
    for graph in (False, True):
        with gpu_problem(c, lattice, shape, precision=precision, schedule=schedule) as gp:
            gp.init_fields(rho)
            for n in (3, 3, 4, 4, 1):
                (gp.step_graph if graph else gp.step)(n)
            assert gp.step_count() == 15
            out.append(gp.get_state())
    assert np.array_equal(out[0], out[1])



@pytest.mark.parametrize("precision,schedule,lattice,shape,kernels", [
    (FP32DEV, FUSED, 0, (1, 40, 130), ("k_mu32", "k_fused32")),
    (FP32, FUSED, 0, (1, 40, 130), ("k_fused32",)),
    (FP32DEV, MULTIPASS, 1, (10, 12, 14), ("k_mp_mu", "k_mp_collide", "k_mp_update"))],
    ids=["fp32dev-fused", "fp32-fused", "fp32dev-multipass-d3q19"])
def test_kernel_timing(precision, schedule, lattice, shape, kernels):
    """lbm_timing_*: one event pair per launch of every kernel of the step
    (8 steps: 6 by lbm_step, 2 by lbm_step_graph, which runs as lbm_step while
    timing), a positive time for each, nothing else recorded, and the same
    state as without timing."""
    c = seeded_mixture(331, 3, lattice, shape)
    rho = smooth_rho(331, c, shape)
    out = []
    for timed in (False, True):
        with gpu_problem(c, lattice, shape, precision=precision, schedule=schedule) as gp:
            gp.init_fields(rho)
            gp.step(1)  # the first step times the launch geometries (not recorded)
            if timed:
                gp.timing_enable(True)
            gp.step(6)
            gp.step_graph(2)
            if timed:
                t = gp.timing_read()
                assert len(t) == len(kernels), t
                for k in kernels:
                    launches, ms = next(v for n, v in t.items() if n.startswith(k))
                    assert launches == 8 and ms > 0.0, (k, t)
                gp.timing_enable(False)
            out.append(gp.get_state())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("precision,schedule,lattice,shape", [
    (FP32DEV, FUSED, 0, (1, 20, 30)), (FP64, FUSED, 0, (1, 12, 30)), (FP64, THREEPASS, 1, (4, 5, 6)),
    (FP32DEV, MULTIPASS, 1, (4, 5, 6))],
    ids=["fp32dev-fused", "fp64-fused", "fp64-threepass-d3q19", "fp32dev-multipass-d3q19"])
def test_density_only_moments(precision, schedule, lattice, shape):
    """lbm_moments with only rho requested (the densities-only kernel, no
    equation of state) returns the densities of the full request bitwise,
    also into a caller's array."""
    c = seeded_mixture(332, 3, lattice, shape)
    rho = smooth_rho(332, c, shape)
    with gpu_problem(c, lattice, shape, precision=precision, schedule=schedule) as gp:
        gp.init_fields(rho)
        gp.step(5)
        full = gp.moments()["rho"]
        only = gp.moments(("rho",))["rho"]
        into = np.empty(full.size)
        gp.moments(("rho",), out_arrays={"rho": into})
    assert np.array_equal(full, only)
    assert np.array_equal(full.reshape(-1), into)
