"""Python binding of ``liblbmfug.so`` (the C ABI of include/lbmfug.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Host arrays are numpy float64 arrays; device buffers are
torch CUDA tensors (PyTorch provides device memory and streams, nothing
else).  Importing this module raises if the library has not been built:
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbmfug.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2306_10652_gb300/build.py "
                      "(or __graft_entry__.build()); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP64, LBM_FP32DEV, LBM_FP32 = 0, 1, 2
LBM_SCHED_AUTO, LBM_SCHED_THREEPASS, LBM_SCHED_FUSED, LBM_SCHED_MULTIPASS = 0, 1, 2, 3
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE, LBM_ENOTSUP = \
    0, -1, -2, -3, -4, -5, -6, -7
LBM_MAX_NC = 16

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class lbm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("schedule", ctypes.c_int),
                ("kappa_ref", ctypes.c_double), ("kappa_ref_index", ctypes.c_int),
                ("M", _dp), ("R", ctypes.c_double), ("stream", _vp), ("monitor_every", ctypes.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", _vp),
                ("tune", ctypes.c_int), ("strip", ctypes.c_int), ("seg_h", ctypes.c_int)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("lbm_options_default", ctypes.c_int, ctypes.POINTER(lbm_options))
_sig("lbm_create", ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
     ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double)
_sig("lbm_set_options", ctypes.c_int, _vp, ctypes.POINTER(lbm_options))
_sig("lbm_init_fields", ctypes.c_int, _vp, _dp, _dp)
_sig("lbm_init_fields_device", ctypes.c_int, _vp, _vp, _vp)
_sig("lbm_step", ctypes.c_int, _vp, ctypes.c_longlong)
_sig("lbm_step_graph", ctypes.c_int, _vp, ctypes.c_longlong)
_sig("lbm_moments", ctypes.c_int, _vp, _dp, _dp, _dp, _dp)
_sig("lbm_moments_device", ctypes.c_int, _vp, _vp, _vp, _vp, _vp)
_sig("lbm_mass", ctypes.c_int, _vp, _dp)
_sig("lbm_forces", ctypes.c_int, _vp, _dp, _dp)
_sig("lbm_schedule_info", ctypes.c_int, _vp, _ip, _ip, _ip, _ip, _ip)
_sig("lbm_convergence", ctypes.c_int, _vp, _dp)
_sig("lbm_get_state", ctypes.c_int, _vp, _dp, ctypes.POINTER(ctypes.c_size_t))
_sig("lbm_set_state", ctypes.c_int, _vp, _dp, ctypes.c_size_t)
_sig("lbm_step_count", ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_longlong))
_sig("lbm_monitor", ctypes.c_int, _vp, _dp, ctypes.POINTER(ctypes.c_longlong), _ip)
_sig("lbm_launch_count", ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_longlong))


class lbm_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


_sig("lbm_timing_enable", ctypes.c_int, _vp, ctypes.c_int)
_sig("lbm_timing_read", ctypes.c_int, _vp, ctypes.POINTER(lbm_kernel_time), ctypes.c_int, _ip)
_sig("lbm_field_sums_noalloc", ctypes.c_int, _vp, ctypes.c_int, ctypes.c_longlong, _vp, _vp, _vp)
class lbm_job(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("T", ctypes.c_double), ("rho", _dp)]


_sig("lbm_batch_create", ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double,
     ctypes.POINTER(lbm_options), ctypes.POINTER(lbm_job), ctypes.c_int)
_sig("lbm_batch_run", ctypes.c_int, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double, _ip)
_sig("lbm_batch_job_state", ctypes.c_int, _vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong), _dp, _ip)
_sig("lbm_batch_info", ctypes.c_int, _vp, _ip, _ip, ctypes.POINTER(ctypes.c_longlong),
     ctypes.POINTER(ctypes.c_longlong))
_sig("lbm_batch_set_threads", ctypes.c_int, _vp, ctypes.c_int)
_sig("lbm_batch_destroy", ctypes.c_int, _vp)
class lbm_request(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Nc", ctypes.c_int), ("a", _dp), ("b", _dp), ("omega", _dp), ("kij", _dp), ("M", _dp),
                ("T", ctypes.c_double), ("tau", ctypes.c_double), ("kappa_ref", ctypes.c_double),
                ("rho", _dp), ("precision", ctypes.c_int), ("check_every", ctypes.c_int),
                ("max_steps", ctypes.c_longlong), ("tol", ctypes.c_double)]


_sig("lbm_server_estimate_bytes", ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
     ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t))
_sig("lbm_server_create", ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_double, ctypes.c_int)
_sig("lbm_server_submit", ctypes.c_int, _vp, ctypes.POINTER(lbm_request), ctypes.POINTER(ctypes.c_longlong))
_sig("lbm_server_poll", ctypes.c_int, _vp, ctypes.c_longlong, _ip, ctypes.POINTER(ctypes.c_longlong), _dp, _dp)
_sig("lbm_server_result", ctypes.c_int, _vp, ctypes.c_longlong, _dp)
_sig("lbm_server_wait_all", ctypes.c_int, _vp)
_sig("lbm_server_stats", ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
     ctypes.POINTER(ctypes.c_size_t), _dp, ctypes.POINTER(ctypes.c_longlong))
_sig("lbm_server_admission", ctypes.c_int, _vp, _ip, ctypes.POINTER(ctypes.c_longlong))
_sig("lbm_server_times", ctypes.c_int, _vp, ctypes.c_longlong, _dp, _dp)
_sig("lbm_server_destroy", ctypes.c_int, _vp)
_sig("lbm_synchronize", ctypes.c_int, _vp)
_sig("lbm_destroy", ctypes.c_int, _vp)
_sig("lbm_lattice_velocities", ctypes.c_int, ctypes.c_int, _ip, _ip, _ip)
_sig("lbm_strerror", ctypes.c_char_p, ctypes.c_int)

EXPORTED = ["lbm_options_default", "lbm_create", "lbm_set_options", "lbm_init_fields",
            "lbm_init_fields_device", "lbm_step", "lbm_moments", "lbm_moments_device", "lbm_mass",
            "lbm_convergence", "lbm_get_state", "lbm_set_state", "lbm_step_count", "lbm_monitor",
            "lbm_launch_count", "lbm_timing_enable", "lbm_timing_read", "lbm_step_graph",
            "lbm_forces", "lbm_schedule_info", "lbm_field_sums_noalloc", "lbm_batch_create", "lbm_batch_run",
            "lbm_batch_job_state", "lbm_batch_info", "lbm_batch_set_threads", "lbm_batch_destroy",
            "lbm_server_estimate_bytes", "lbm_server_create", "lbm_server_submit", "lbm_server_poll",
            "lbm_server_result", "lbm_server_wait_all", "lbm_server_stats", "lbm_server_admission",
            "lbm_server_times", "lbm_server_destroy",
            "lbm_synchronize", "lbm_destroy", "lbm_lattice_velocities", "lbm_strerror"]


class LbmError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {lbm_strerror(status)} ({status})")


def lbm_strerror(status: int) -> str:
    return _lib.lbm_strerror(int(status)).decode()


def _check(st, where):
    if st != LBM_OK:
        raise LbmError(st, where)


def _host(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _hp(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _dev(t):
    """Raw device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise ValueError("device buffers must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def lbm_field_sums_noalloc(d_field, nc, n, d_out, d_nonfinite=None, stream=None):
    """Per-component sums of a device field[nc][n] into device out[nc], with no
    device allocation (see the C declaration).  Device buffers are torch CUDA
    tensors (float64 field and out, int32 flag); stream is a raw cudaStream_t."""
    if d_nonfinite is not None and not (d_nonfinite.is_cuda and str(d_nonfinite.dtype) == "torch.int32"):
        raise ValueError("d_nonfinite must be an int32 CUDA tensor")
    _check(_lib.lbm_field_sums_noalloc(_dev(d_field), int(nc), int(n), _dev(d_out),
                                       None if d_nonfinite is None else ctypes.c_void_p(d_nonfinite.data_ptr()),
                                       None if stream is None else ctypes.c_void_p(int(stream))),
           "lbm_field_sums_noalloc")


def lbm_lattice_velocities(lattice: int):
    D, Q = ctypes.c_int(), ctypes.c_int()
    e = np.zeros((19, 3), dtype=np.int32)
    _check(_lib.lbm_lattice_velocities(lattice, ctypes.byref(D), ctypes.byref(Q),
                                       e.ctypes.data_as(_ip)), "lbm_lattice_velocities")
    return D.value, Q.value, e[:Q.value].copy()


class Problem:
    """One periodic problem (a handle of the C ABI).

    ``Problem(lattice, nx, ny, nz, a, b, omega, kij, T, tau, **options)``
    mirrors ``lbm_create`` + ``lbm_set_options``; option keywords are the
    fields of ``lbm_options`` (precision, schedule, kappa_ref,
    kappa_ref_index, M, R, stream).
    """

    def __init__(self, lattice, nx, ny, nz, a, b, omega, kij=None, T=None, tau=1.0, *,
                 precision=LBM_FP64, schedule=LBM_SCHED_AUTO, kappa_ref=0.02, kappa_ref_index=0,
                 M=None, R=1.0, stream=None, monitor_every=0, tune=1, strip=0, seg_h=0):
        self._h = None
        a = _host(a)
        nc = a.size
        self.lattice, self.nx, self.ny, self.nz, self.nc = int(lattice), int(nx), int(ny), int(nz), nc
        self.D, self.Q, self.e = lbm_lattice_velocities(self.lattice)
        self.precision = precision
        b = _host(b, nc)
        omega = _host(omega, nc)
        kij = None if kij is None else _host(kij, nc * nc)
        h = _vp()
        _check(_lib.lbm_create(ctypes.byref(h), self.lattice, self.nx, self.ny, self.nz, nc,
                               _hp(a), _hp(b), _hp(omega), _hp(kij), float(T), float(tau)),
               "lbm_create")
        self._h = h
        opt = lbm_options()
        _lib.lbm_options_default(ctypes.byref(opt))
        opt.precision = int(precision)
        opt.schedule = int(schedule)
        opt.kappa_ref = float(kappa_ref)
        opt.kappa_ref_index = int(kappa_ref_index)
        self._M = None if M is None else _host(M, nc)
        opt.M = _hp(self._M)
        opt.R = float(R)
        opt.stream = None if stream is None else ctypes.c_void_p(int(stream))
        opt.monitor_every = int(monitor_every)
        opt.tune = int(tune)
        opt.strip = int(strip)
        opt.seg_h = int(seg_h)
        _check(_lib.lbm_set_options(self._h, ctypes.byref(opt)), "lbm_set_options")

    # -- shapes --
    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    # -- calls --
    def init_fields(self, rho, u=None):
        rho = _host(rho, self.nc * self.N)
        u = None if u is None else _host(u, self.D * self.N)
        _check(_lib.lbm_init_fields(self._h, _hp(rho), _hp(u)), "lbm_init_fields")

    def init_fields_device(self, d_rho, d_u=None):
        _check(_lib.lbm_init_fields_device(self._h, _dev(d_rho), _dev(d_u)), "lbm_init_fields_device")

    def step(self, n=1):
        _check(_lib.lbm_step(self._h, int(n)), "lbm_step")

    def step_graph(self, n):
        """lbm_step_graph: n steps replayed from a captured CUDA graph."""
        _check(_lib.lbm_step_graph(self._h, int(n)), "lbm_step_graph")

    def moments(self, want=("rho", "u", "p", "lnf"), out_arrays=None):
        """lbm_moments of the fields in `want`; out_arrays may give float64
        C-contiguous host arrays (for example pinned) to write them into."""
        out = {}
        given = out_arrays or {}

        def buf(name, shape):
            if name not in want:
                return None
            if name in given:
                a = given[name]
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != int(np.prod(shape)):
                    raise ValueError(f"out_arrays[{name!r}]: float64 C-contiguous with {int(np.prod(shape))} values")
                return a.reshape(shape)
            return np.empty(shape)

        rho = buf("rho", (self.nc,) + self.shape)
        u = buf("u", (self.D,) + self.shape)
        p = buf("p", self.shape)
        lnf = buf("lnf", (self.nc,) + self.shape)
        _check(_lib.lbm_moments(self._h, _hp(rho), _hp(u), _hp(p), _hp(lnf)), "lbm_moments")
        for k, v in (("rho", rho), ("u", u), ("p", p), ("lnf", lnf)):
            if v is not None:
                out[k] = v
        return out

    def moments_device(self, d_rho=None, d_u=None, d_p=None, d_lnf=None):
        _check(_lib.lbm_moments_device(self._h, _dev(d_rho), _dev(d_u), _dev(d_p), _dev(d_lnf)),
               "lbm_moments_device")

    def mass(self):
        m = np.empty(self.nc)
        _check(_lib.lbm_mass(self._h, _hp(m)), "lbm_mass")
        return m

    def forces(self, want=("F", "mu")):
        """{"F": [Nc, 2, nz, ny, nx], "mu": [Nc, nz, ny, nx]} (lbm_forces, D2Q9)."""
        F = np.empty((self.nc, 2) + self.shape) if "F" in want else None
        mu = np.empty((self.nc,) + self.shape) if "mu" in want else None
        _check(_lib.lbm_forces(self._h, _hp(F), _hp(mu)), "lbm_forces")
        return {k: v for k, v in (("F", F), ("mu", mu)) if v is not None}

    def schedule_info(self):
        """dict(fused, strip, nstrips, seg_h, segs) of the step's launch geometry."""
        v = [ctypes.c_int() for _ in range(5)]
        _check(_lib.lbm_schedule_info(self._h, *[ctypes.byref(x) for x in v]), "lbm_schedule_info")
        return dict(zip(("fused", "strip", "nstrips", "seg_h", "segs"), (x.value for x in v)))

    def convergence(self):
        v = ctypes.c_double()
        _check(_lib.lbm_convergence(self._h, ctypes.byref(v)), "lbm_convergence")
        return v.value

    def get_state(self):
        n = ctypes.c_size_t()
        _check(_lib.lbm_get_state(self._h, None, ctypes.byref(n)), "lbm_get_state")
        buf = np.empty(n.value // 8)
        _check(_lib.lbm_get_state(self._h, _hp(buf), ctypes.byref(n)), "lbm_get_state")
        return buf.reshape((self.nc, self.Q) + self.shape)

    def set_state(self, g):
        g = _host(g, self.nc * self.Q * self.N)
        _check(_lib.lbm_set_state(self._h, _hp(g), g.nbytes), "lbm_set_state")

    def monitor(self):
        """(mass[Nc] or None, step it was taken at, nonfinite flag)."""
        m = np.empty(self.nc)
        at = ctypes.c_longlong()
        nf = ctypes.c_int()
        _check(_lib.lbm_monitor(self._h, _hp(m), ctypes.byref(at), ctypes.byref(nf)), "lbm_monitor")
        return (m if at.value >= 0 else None), at.value, bool(nf.value)

    def launch_count(self):
        v = ctypes.c_longlong()
        _check(_lib.lbm_launch_count(self._h, ctypes.byref(v)), "lbm_launch_count")
        return v.value

    def timing_enable(self, on=True):
        """lbm_timing_enable: CUDA events around every kernel launch of lbm_step."""
        _check(_lib.lbm_timing_enable(self._h, 1 if on else 0), "lbm_timing_enable")

    def timing_read(self):
        """lbm_timing_read: {kernel name: (launches, total ms)} since timing was enabled."""
        buf = (lbm_kernel_time * 16)()
        n = ctypes.c_int()
        _check(_lib.lbm_timing_read(self._h, buf, 16, ctypes.byref(n)), "lbm_timing_read")
        return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms)) for k in range(min(n.value, 16))}

    def step_count(self):
        v = ctypes.c_longlong()
        _check(_lib.lbm_step_count(self._h, ctypes.byref(v)), "lbm_step_count")
        return v.value

    def synchronize(self):
        _check(_lib.lbm_synchronize(self._h), "lbm_synchronize")

    def close(self):
        if self._h is not None:
            _lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many small D2Q9 problems advanced together (the lbm_batch_* calls).

    ``jobs`` is a list of (T, rho[Nc, ny, nx]) pairs; the components' PR
    parameters, tau and the options are shared.
    """

    def __init__(self, a, b, omega, kij, tau, jobs, *, precision=LBM_FP32, kappa_ref=0.02,
                 kappa_ref_index=0, M=None, R=1.0, stream=None):
        self._h = None
        a = _host(a)
        self.nc = a.size
        b = _host(b, self.nc)
        omega = _host(omega, self.nc)
        kij = None if kij is None else _host(kij, self.nc * self.nc)
        opt = lbm_options()
        _lib.lbm_options_default(ctypes.byref(opt))
        opt.precision = int(precision)
        opt.kappa_ref = float(kappa_ref)
        opt.kappa_ref_index = int(kappa_ref_index)
        self._M = None if M is None else _host(M, self.nc)
        opt.M = _hp(self._M)
        opt.R = float(R)
        opt.stream = None if stream is None else ctypes.c_void_p(int(stream))
        self._rho = []
        arr = (lbm_job * len(jobs))()
        self.shapes = []
        for k, (T, rho) in enumerate(jobs):
            r = np.ascontiguousarray(rho, dtype=np.float64)
            ny, nx = r.shape[-2], r.shape[-1]
            r = r.reshape(self.nc, ny, nx)
            self._rho.append(r)
            self.shapes.append((ny, nx))
            arr[k].nx, arr[k].ny, arr[k].T = nx, ny, float(T)
            arr[k].rho = r.ctypes.data_as(_dp)
        h = _vp()
        _check(_lib.lbm_batch_create(ctypes.byref(h), self.nc, _hp(a), _hp(b), _hp(omega), _hp(kij),
                                     float(tau), ctypes.byref(opt), arr, len(jobs)), "lbm_batch_create")
        self._h = h
        self._rho = None
        self.njobs = len(jobs)

    def run(self, max_steps, check_every=1000, tol=1e-10):
        n = ctypes.c_int()
        _check(_lib.lbm_batch_run(self._h, int(max_steps), int(check_every), float(tol), ctypes.byref(n)),
               "lbm_batch_run")
        return n.value

    def state(self, job):
        ny, nx = self.shapes[job]
        rho = np.empty((self.nc, ny, nx))
        steps = ctypes.c_longlong()
        d = ctypes.c_double()
        c = ctypes.c_int()
        _check(_lib.lbm_batch_job_state(self._h, int(job), _hp(rho), ctypes.byref(steps), ctypes.byref(d),
                                        ctypes.byref(c)), "lbm_batch_job_state")
        return {"rho": rho, "steps": steps.value, "last_drho": d.value, "converged": c.value == 1,
                "failed": c.value == 2}

    def info(self):
        th, ct = ctypes.c_int(), ctypes.c_int()
        rd, ln = ctypes.c_longlong(), ctypes.c_longlong()
        _check(_lib.lbm_batch_info(self._h, ctypes.byref(th), ctypes.byref(ct), ctypes.byref(rd),
                                   ctypes.byref(ln)), "lbm_batch_info")
        return {"threads": th.value, "ctas": ct.value, "rounds": rd.value, "launches": ln.value}

    def set_threads(self, threads):
        _check(_lib.lbm_batch_set_threads(self._h, int(threads)), "lbm_batch_set_threads")

    def close(self):
        if self._h is not None:
            _lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Admission-controlled request loop (the lbm_server_* calls)."""

    STATES = {0: "queued", 1: "running", 2: "converged", 3: "failed", 4: "exhausted"}

    def __init__(self, hbm_budget_frac=0.8, max_active=8):
        h = _vp()
        _check(_lib.lbm_server_create(ctypes.byref(h), float(hbm_budget_frac), int(max_active)),
               "lbm_server_create")
        self._h = h
        self._shapes = {}

    def submit(self, lattice, a, b, omega, kij, T, tau, rho, *, precision=LBM_FP32DEV, check_every=1000,
               max_steps=100000, tol=1e-10, M=None, kappa_ref=0.02):
        a = _host(a)
        nc = a.size
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        shape = rho.shape[1:] if rho.ndim == 4 else (1,) + rho.shape[1:]
        nz, ny, nx = shape
        keep = [a, _host(b, nc), _host(omega, nc), None if kij is None else _host(kij, nc * nc),
                None if M is None else _host(M, nc), rho.reshape(-1)]
        q = lbm_request(lattice=int(lattice), nx=nx, ny=ny, nz=nz, Nc=nc, a=_hp(keep[0]), b=_hp(keep[1]),
                        omega=_hp(keep[2]), kij=_hp(keep[3]), M=_hp(keep[4]), T=float(T), tau=float(tau),
                        kappa_ref=float(kappa_ref), rho=_hp(keep[5]), precision=int(precision),
                        check_every=int(check_every), max_steps=int(max_steps), tol=float(tol))
        jid = ctypes.c_longlong()
        _check(_lib.lbm_server_submit(self._h, ctypes.byref(q), ctypes.byref(jid)), "lbm_server_submit")
        self._shapes[jid.value] = (nc,) + tuple(shape)
        return jid.value

    def poll(self, jid):
        st, steps = ctypes.c_int(), ctypes.c_longlong()
        lat, d = ctypes.c_double(), ctypes.c_double()
        rc = _lib.lbm_server_poll(self._h, int(jid), ctypes.byref(st), ctypes.byref(steps), ctypes.byref(lat),
                                  ctypes.byref(d))
        if rc == LBM_EINVAL:
            raise LbmError(rc, "lbm_server_poll")
        return {"state": self.STATES[st.value], "steps": steps.value, "latency_s": lat.value,
                "last_drho": d.value, "status": rc}

    def result(self, jid):
        rho = np.empty(self._shapes[jid])
        _check(_lib.lbm_server_result(self._h, int(jid), _hp(rho)), "lbm_server_result")
        return rho

    def wait_all(self):
        _check(_lib.lbm_server_wait_all(self._h), "lbm_server_wait_all")

    def stats(self):
        sub, comp, rd = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        peak, bud = ctypes.c_size_t(), ctypes.c_double()
        _check(_lib.lbm_server_stats(self._h, ctypes.byref(sub), ctypes.byref(comp), ctypes.byref(peak),
                                     ctypes.byref(bud), ctypes.byref(rd)), "lbm_server_stats")
        return {"submitted": sub.value, "completed": comp.value, "peak_bytes": peak.value,
                "budget_bytes": bud.value, "rounds": rd.value}

    def admission(self):
        """{"peak_active", "memory_waits"} (lbm_server_admission)."""
        pa, mw = ctypes.c_int(), ctypes.c_longlong()
        _check(_lib.lbm_server_admission(self._h, ctypes.byref(pa), ctypes.byref(mw)), "lbm_server_admission")
        return {"peak_active": pa.value, "memory_waits": mw.value}

    def times(self, jid):
        """(queued seconds, running seconds) of a finished request (lbm_server_times)."""
        q, r = ctypes.c_double(), ctypes.c_double()
        _check(_lib.lbm_server_times(self._h, int(jid), ctypes.byref(q), ctypes.byref(r)), "lbm_server_times")
        return q.value, r.value

    def close(self):
        if self._h is not None:
            _lib.lbm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def lbm_server_estimate_bytes(lattice, nx, ny, nz, nc, precision):
    v = ctypes.c_size_t()
    _check(_lib.lbm_server_estimate_bytes(int(lattice), int(nx), int(ny), int(nz), int(nc), int(precision),
                                          ctypes.byref(v)), "lbm_server_estimate_bytes")
    return v.value
