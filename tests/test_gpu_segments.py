"""Element-wise oracle parity of the fused kernels on multi-row segments.

The fused D2Q9 kernels walk a segment of rows per CTA, carrying ring buffers
of density, psi and mu rows and the density pairs of the rows being updated
from one row to the next.  The shapes here are tall enough that the launch
geometry gives each CTA at least eight rows (asserted through
lbm_schedule_info, so a change of geometry cannot shrink it unnoticed).
Every population is compared with the oracle after two or three steps.

Tolerances, per component relative to max |g_i|: binary64 storage 1e-12
(the two sides differ only in the order of roundings, about 1e-16 per
operation over a few hundred operations per node-step); binary32 storage
2e-6 (a stored population carries one binary32 rounding, 2^-24 = 6e-8 of
its size, per step, and the forcing/equilibrium terms a few more; the rest
population and densities are exact pairs); binary32 thermodynamics 1e-5
(ln f_i from hardware logarithms with absolute error 2^-21.4, times RT,
enters the force through differences).
"""
from __future__ import annotations

import numpy as np
import pytest

from helpers import gpu_problem, oracle_problem, order_map, seeded_mixture, smooth_rho
from paper_2306_10652_gb300 import synth

pytestmark = pytest.mark.gpu

FP64, FP32DEV, FP32 = 0, 1, 2
TOL = {FP64: 1e-12, FP32DEV: 2e-6, FP32: 1e-5}

SEG_CASES = [
    # seed, nc, shape (nz, ny, nx), steps
    (101, 3, (1, 4096, 130), 3),
    (102, 10, (1, 1216, 250), 2),
]
_ref = {}


def reference(case):
    if case not in _ref:
        seed, nc, shape, steps = case
        c = seeded_mixture(seed, nc, 0, shape)
        M = synth.uniform(seed, 0.5, 2.0, nc)
        orc = oracle_problem(c, 0, shape, tau=0.9, M=M)
        rho = smooth_rho(seed, c, shape, 0.05, 0.4) * M[:, None, None, None]
        u = synth.random_velocity(seed, 2, shape, 1e-3)
        _ref[case] = (c, M, rho, u, orc.step(orc.init_equilibrium(rho, u), steps))
    return _ref[case]


@pytest.mark.parametrize("precision", [FP64, FP32DEV, FP32], ids=["fp64", "fp32dev", "fp32"])
@pytest.mark.parametrize("case", SEG_CASES, ids=lambda c: f"nc{c[1]}-{c[2][1]}x{c[2][2]}")
def test_fused_multirow_segments(case, precision):
    seed, nc, shape, steps = case
    c, M, rho, u, g_ref = reference(case)
    with gpu_problem(c, 0, shape, tau=0.9, M=M, precision=precision, schedule=2) as gp:
        gp.init_fields(rho, u)
        info = gp.schedule_info()
        assert info["fused"] == 1 and info["seg_h"] >= 8 and info["segs"] >= 2, info
        gp.step(steps)
        g = gp.get_state()[:, order_map(0, gp.e)]
    scale = np.abs(g_ref).max(axis=(1, 2, 3, 4), keepdims=True)
    err = float((np.abs(g - g_ref) / scale).max())
    assert err < TOL[precision], (err, info)
