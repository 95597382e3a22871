"""The C ABI: the library builds, loads, exports every declared symbol, and
validates arguments without touching a GPU."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_10652_gb300.build import build
    build()
    from paper_2306_10652_gb300 import lbmfug
    return lbmfug


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbm\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lbm_step" in names and "lbm_create" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    names = declared_functions()
    assert set(lib.EXPORTED) <= names


def _create(lib, **kw):
    args = dict(lattice=0, nx=4, ny=4, nz=1, a=[0.04, 0.05], b=[0.09, 0.1], omega=[0.1, 0.2],
                kij=[0.0, 0.05, 0.05, 0.0], T=0.06, tau=1.0)
    args.update(kw)
    a = np.asarray(args["a"], float)
    nc = len(a)
    h = ctypes.c_void_p()
    kij = None if args["kij"] is None else np.asarray(args["kij"], float)
    st = lib._lib.lbm_create(ctypes.byref(h), args["lattice"], args["nx"], args["ny"], args["nz"], nc,
                             a.ctypes.data_as(lib._dp),
                             np.asarray(args["b"], float).ctypes.data_as(lib._dp),
                             np.asarray(args["omega"], float).ctypes.data_as(lib._dp),
                             None if kij is None else kij.ctypes.data_as(lib._dp),
                             float(args["T"]), float(args["tau"]))
    if h.value:
        lib._lib.lbm_destroy(h)
    return st


def test_create_validates(lib):
    assert _create(lib) == lib.LBM_OK
    assert _create(lib, kij=None) == lib.LBM_OK
    assert _create(lib, lattice=2) == lib.LBM_EINVAL
    assert _create(lib, nz=2) == lib.LBM_EINVAL           # D2Q9 needs nz = 1
    assert _create(lib, lattice=1, nz=3) == lib.LBM_OK
    assert _create(lib, nx=0) == lib.LBM_EINVAL
    assert _create(lib, tau=0.5) == lib.LBM_EINVAL
    assert _create(lib, T=0.0) == lib.LBM_EINVAL
    assert _create(lib, T=float("nan")) == lib.LBM_EINVAL
    assert _create(lib, a=[0.04, -0.05]) == lib.LBM_EINVAL
    assert _create(lib, b=[0.0, 0.1]) == lib.LBM_EINVAL
    assert _create(lib, kij=[0.0, 0.05, 0.06, 0.0]) == lib.LBM_EINVAL   # not symmetric
    assert _create(lib, kij=[0.1, 0.05, 0.05, 0.0]) == lib.LBM_EINVAL   # nonzero diagonal
    assert _create(lib, kij=[0.0, 1.0, 1.0, 0.0]) == lib.LBM_EINVAL     # |k| >= 1
    assert _create(lib, a=[0.04] * 17, b=[0.1] * 17, omega=[0.1] * 17, kij=None) == lib.LBM_EINVAL


def test_options_validate_and_states(lib):
    p = lib.Problem(0, 4, 4, 1, [0.04], [0.1], [0.1], None, 0.06, 1.0)
    opt = lib.lbm_options()
    lib._lib.lbm_options_default(ctypes.byref(opt))
    assert opt.kappa_ref == 0.02 and opt.R == 1.0 and opt.precision == lib.LBM_FP64
    bad = lib.lbm_options()
    lib._lib.lbm_options_default(ctypes.byref(bad))
    bad.precision = 7
    assert lib._lib.lbm_set_options(p._h, ctypes.byref(bad)) == lib.LBM_EINVAL
    bad.precision = 0
    bad.kappa_ref_index = 3
    assert lib._lib.lbm_set_options(p._h, ctypes.byref(bad)) == lib.LBM_EINVAL
    # stepping before initialisation is a state error, not a crash
    assert lib._lib.lbm_step(p._h, 1) == lib.LBM_ESTATE
    assert lib._lib.lbm_step(p._h, -1) == lib.LBM_EINVAL
    with pytest.raises(lib.LbmError):
        p.init_fields(np.full(16, -1.0))      # non-positive density rejected on the host
    assert lib._lib.lbm_destroy(None) == lib.LBM_OK
    p.close()


def test_strerror_and_lattice_tables(lib):
    assert lib.lbm_strerror(lib.LBM_EINVAL) == "invalid argument"
    assert lib.lbm_strerror(12345) == "unknown status"
    for lat, (D, Q) in ((0, (2, 9)), (1, (3, 19))):
        d, q, e = lib.lbm_lattice_velocities(lat)
        assert (d, q) == (D, Q)
        assert (e[0] == 0).all()
        # opposite pairs (2k-1, 2k) and every vector distinct
        for k in range(1, Q, 2):
            assert (e[k] == -e[k + 1]).all()
        assert len({tuple(v) for v in e}) == Q


def test_timing_arguments_and_states(lib):
    p = lib.Problem(0, 4, 4, 1, [0.04], [0.1], [0.1], None, 0.06, 1.0)
    buf = (lib.lbm_kernel_time * 4)()
    n = ctypes.c_int(7)
    # reading before enabling is a state error; bad arguments are rejected
    assert lib._lib.lbm_timing_read(p._h, buf, 4, ctypes.byref(n)) == lib.LBM_ESTATE
    assert n.value == 0
    assert lib._lib.lbm_timing_enable(p._h, 2) == lib.LBM_EINVAL
    assert lib._lib.lbm_timing_enable(None, 1) == lib.LBM_EINVAL
    assert lib._lib.lbm_timing_read(p._h, None, 4, ctypes.byref(n)) == lib.LBM_EINVAL
    assert lib._lib.lbm_timing_read(p._h, buf, -1, ctypes.byref(n)) == lib.LBM_EINVAL
    # enabled before any step: nothing has launched yet
    p.timing_enable(True)
    assert p.timing_read() == {}
    p.timing_enable(False)
    assert lib._lib.lbm_timing_read(p._h, buf, 4, ctypes.byref(n)) == lib.LBM_ESTATE
    p.close()


def test_init_fields_rejects_bad_values_in_large_fields(lib):
    """The host validation of lbm_init_fields splits large fields over host
    threads; a bad value in any part is still rejected before any device work."""
    nx = ny = 2048  # 4,194,304 values: the threaded path
    p = lib.Problem(0, nx, ny, 1, [0.04], [0.1], [0.1], None, 0.06, 1.0)
    rho = np.full(nx * ny, 0.5)
    for k in (0, nx * ny // 3, nx * ny - 1):
        bad = rho.copy()
        bad[k] = -1.0 if k % 2 == 0 else float("nan")
        st = lib._lib.lbm_init_fields(p._h, bad.ctypes.data_as(lib._dp), None)
        assert st == lib.LBM_EINVAL, (k, st)
    p.close()
