"""The allocation-free field sums (lbm_field_sums_noalloc) against lbm_mass.

lbm_field_sums_noalloc serves callers that cannot allocate device memory
where they need a reduction; it keeps its partial sums in a scratch area
built into the library.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from helpers import gpu_problem, seeded_mixture, smooth_rho

pytestmark = pytest.mark.gpu


def test_noalloc_sums_match_mass_twice():
    import torch

    from paper_2306_10652_gb300 import lbmfug

    shape = (1, 61, 203)
    nc = 4
    c = seeded_mixture(91, nc, 0, shape)
    rho = smooth_rho(91, c, shape)
    with gpu_problem(c, 0, shape) as gp:
        gp.init_fields(rho)
        ref = gp.mass()                     # the existing entry point
        d_field = torch.empty(nc * gp.N, dtype=torch.float64, device="cuda")
        gp.moments_device(d_rho=d_field)    # the same densities, on the device
        gp.synchronize()
    stream = torch.cuda.current_stream()
    for _ in range(2):                      # two calls in a row share the scratch
        out = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
        flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        lbmfug.lbm_field_sums_noalloc(d_field, nc, gp.N, out, flag, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert int(flag.item()) == 0
        # the tolerance of the binary64 mass tests; the summation order is the same
        assert np.allclose(got, ref, rtol=1e-13, atol=0), (got, ref)


def test_noalloc_rejects_beyond_capacity():
    import torch

    from paper_2306_10652_gb300 import lbmfug

    field = torch.ones(17 * 8, dtype=torch.float64, device="cuda")
    out = torch.empty(17, dtype=torch.float64, device="cuda")
    with pytest.raises(lbmfug.LbmError) as e:
        lbmfug.lbm_field_sums_noalloc(field, 17, 8, out)
    assert e.value.status == lbmfug.LBM_EINVAL
