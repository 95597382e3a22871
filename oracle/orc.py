"""ctypes binding of the C oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays use the
oracle's layout: populations ``g[i, a, z, y, x]`` in the post-streaming
convention of Eq. (1a), fields ``rho[i, z, y, x]``, ``u[d, z, y, x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build_oracle(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``_build/liboracle.so`` (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_problem_size.restype = ctypes.c_int
            lib.orc_problem_set.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int]
            lib.orc_eos.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            lib.orc_step.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_longlong]
            lib.orc_moments.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp]
            lib.orc_init_equilibrium.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            lib.orc_mass.argtypes = [ctypes.c_void_p, _dp, _dp]
            lib.orc_gradient.argtypes = [ctypes.c_void_p, _dp, _dp]
            lib.orc_laplacian.argtypes = [ctypes.c_void_p, _dp, _dp]
            lib.orc_alpha.argtypes = [ctypes.c_double] * 5
            lib.orc_alpha.restype = ctypes.c_double
            lib.orc_critical_temperature.argtypes = [ctypes.c_double] * 3
            lib.orc_critical_temperature.restype = ctypes.c_double
            lib.orc_feq_forcing.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
            lib.orc_lattice_info.argtypes = [ctypes.c_int, _ip, _ip, _ip, _dp]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def set_threads(n: int) -> int:
    """Threads of the oracle's node loops (n < 1: every core); returns the count in use.
    Results do not depend on it."""
    return int(_load().orc_set_threads(int(n)))


def lattice_info(lattice: int):
    """(D, Q, e[Q,3] int, w[Q]) of the oracle's lattice tables."""
    lib = _load()
    D, Q = ctypes.c_int(), ctypes.c_int()
    e = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    lib.orc_lattice_info(lattice, ctypes.byref(D), ctypes.byref(Q),
                         e.ctypes.data_as(_ip), _ptr(w))
    return D.value, Q.value, e[:Q.value].copy(), w[:Q.value].copy()


def feq_forcing(lattice: int, rho_i: float, u, F_i, grad_rho_i):
    """Eq. (1b) equilibrium and Eq. (1c) forcing term at one node (one component)."""
    lib = _load()
    u3 = np.zeros(3); u3[:len(u)] = u
    F3 = np.zeros(3); F3[:len(F_i)] = F_i
    G3 = np.zeros(3); G3[:len(grad_rho_i)] = grad_rho_i
    geq = np.zeros(19); Fa = np.zeros(19)
    Q = lib.orc_feq_forcing(lattice, float(rho_i), _ptr(u3), _ptr(F3), _ptr(G3), _ptr(geq), _ptr(Fa))
    return geq[:Q].copy(), Fa[:Q].copy()


class OracleProblem:
    """One periodic problem: lattice, box, Nc components, PR parameters, T, tau."""

    def __init__(self, lattice, nx, ny, nz, a, b, omega, kij=None, T=None, tau=1.0,
                 M=None, R=1.0, kappa_ref=0.02, kappa_ref_index=0):
        lib = _load()
        self.lattice = int(lattice)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.nc = int(self.a.size)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.omega = np.ascontiguousarray(omega, dtype=np.float64)
        self.kij = np.ascontiguousarray(np.zeros((self.nc, self.nc)) if kij is None else kij,
                                        dtype=np.float64)
        self.M = np.ascontiguousarray(np.ones(self.nc) if M is None else M, dtype=np.float64)
        self.T, self.tau, self.R = float(T), float(tau), float(R)
        self.kappa_ref, self.kappa_ref_index = float(kappa_ref), int(kappa_ref_index)
        self.D, self.Q, self.e, self.w = lattice_info(self.lattice)
        self._buf = ctypes.create_string_buffer(lib.orc_problem_size())
        rc = lib.orc_problem_set(self._buf, self.lattice, self.nx, self.ny, self.nz, self.nc,
                                 _ptr(self.a), _ptr(self.b), _ptr(self.omega), _ptr(self.kij.reshape(-1)),
                                 _ptr(self.M), self.T, self.tau, self.R, self.kappa_ref,
                                 self.kappa_ref_index)
        if rc != 0:
            raise ValueError("invalid oracle problem")

    # -- shapes ---------------------------------------------------------
    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    # -- thermodynamics -------------------------------------------------
    def eos(self, rho_molar):
        """(p, ln f[Nc]) from Eqs. (9)-(12) at molar densities rho~_i."""
        lib = _load()
        rm = np.ascontiguousarray(rho_molar, dtype=np.float64)
        p = ctypes.c_double()
        lnf = np.zeros(self.nc)
        if lib.orc_eos(self._buf, _ptr(rm), ctypes.byref(p), _ptr(lnf)) != 0:
            raise ValueError("non-positive total density")
        return p.value, lnf

    def alpha(self):
        lib = _load()
        return np.array([lib.orc_alpha(self.a[i], self.b[i], self.omega[i], self.T, self.R)
                         for i in range(self.nc)])

    def critical_temperatures(self):
        lib = _load()
        return np.array([lib.orc_critical_temperature(self.a[i], self.b[i], self.R)
                         for i in range(self.nc)])

    # -- lattice Boltzmann ----------------------------------------------
    def init_equilibrium(self, rho, u=None):
        lib = _load()
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape((self.nc,) + self.shape)
        g = np.zeros((self.nc, self.Q) + self.shape)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape((self.D,) + self.shape)
        lib.orc_init_equilibrium(self._buf, _ptr(rho), _ptr(uu), _ptr(g))
        return g

    def step(self, g, nsteps=1):
        lib = _load()
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.nc, self.Q) + self.shape)
        out = np.empty_like(g)
        rc = lib.orc_step(self._buf, _ptr(g), _ptr(out), int(nsteps))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")
        return out

    def moments(self, g):
        lib = _load()
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.nc, self.Q) + self.shape)
        rho = np.zeros((self.nc,) + self.shape)
        u = np.zeros((self.D,) + self.shape)
        p = np.zeros(self.shape)
        lnf = np.zeros((self.nc,) + self.shape)
        F = np.zeros((self.nc, self.D) + self.shape)
        rc = lib.orc_moments(self._buf, _ptr(g), _ptr(rho), _ptr(u), _ptr(p), _ptr(lnf), _ptr(F))
        if rc != 0:
            raise RuntimeError(f"oracle moments failed ({rc})")
        return {"rho": rho, "u": u, "p": p, "lnf": lnf, "F": F}

    def mass(self, g):
        lib = _load()
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.nc, self.Q) + self.shape)
        m = np.zeros(self.nc)
        lib.orc_mass(self._buf, _ptr(g), _ptr(m))
        return m

    def gradient(self, X):
        lib = _load()
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(self.shape)
        G = np.zeros((self.D,) + self.shape)
        lib.orc_gradient(self._buf, _ptr(X), _ptr(G))
        return G

    def laplacian(self, X):
        lib = _load()
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(self.shape)
        Y = np.zeros(self.shape)
        lib.orc_laplacian(self._buf, _ptr(X), _ptr(Y))
        return Y
