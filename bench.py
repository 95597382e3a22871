"""Benchmark of the per-step multicomponent LBM hot path on GB300.

Workload (headline): spinodal decomposition, D2Q9 2048 x 2048 periodic,
Nc = 10 seeded Peng-Robinson components (parameters and the uniform state
written by oracle/make_workloads.py into paper_2306_10652_gb300/workloads/),
+-1 % seeded multiplicative density noise.  A step is one full update of
all populations (pull of the paper's Eq. 1a, Eqs. 1b/1c/5/9-12) plus the
on-device per-component mass reduction.

Metric: Nc-weighted lattice updates per second, Nc * nodes * steps / s / 1e9
("Nc*GLUPS"), whole job.  Roofline: algorithmic bytes per node-step
2 * Q * Nc * bytes_per_population (each population read and written once).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--nc NC] [--precision fp32dev|fp64] [--schedule auto|threepass|fused]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_FILE = os.path.join(ROOT, "paper_2306_10652_gb300", "workloads", "spinodal_2048.json")
METRIC = "Nc·GLUPS"
HBM_FALLBACK_GBS = 6800.0


def load_case(nc):
    d = json.load(open(WORKLOAD_FILE))
    case = [c for c in d["cases"] if c["nc"] == nc][0]
    return d, case


def initial_density(d, case, nx, ny, seed=2):
    """rho_i = z_i rho~ M_i (M_i = 1) times the seeded multiplicative noise."""
    from paper_2306_10652_gb300 import synth
    z = np.asarray(case["z"])
    rho = z[:, None, None] * case["rho_molar_total"] * np.ones((1, ny, nx))
    return (rho * synth.multiplicative_noise(seed, rho.shape, 0.01))[:, None]  # [nc, 1, ny, nx]


# DRAM bytes per node of one launch of the dominant kernel (ncu dram__bytes_read
# + dram__bytes_write on a 2048 x 1024 case, larger than L2), keyed on (form,
# schedule, Nc) and on the kernel they were captured from; the traffic is per
# node (strip and segment halos come from L2), so it scales with the nodes of a
# launch.  profiles/fp32dev_mu_pass_and_step_spinodal2048_nc10.md: the step
# kernel k_fused32<10, DF64> moved 1062.2 + 799.0 MB over 2,097,152 nodes.
# A form without an entry, or whose kernel has changed since, reports null.
NCU_TRAFFIC_B_PER_NODE = {
    ("fp32dev", "auto", 10): ("k_fused32<10, DF64> (step kernel)", (1062.237440e6 + 798.856960e6) / 2097152),
}


def traffic_per_launch(args, nc, N):
    v = NCU_TRAFFIC_B_PER_NODE.get((args.precision, args.schedule, nc))
    return (None, None) if v is None else (v[1] * N, v[0])


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, fl in rows for k, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


class BusySampler:
    """nvidia-smi utilization.gpu (percent of time a kernel ran) and memory.used
    (MiB) every 200 ms."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", "--query-gpu=utilization.gpu,memory.used",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.util, self.mem = [], []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()
            for line in open(self.path):
                try:
                    u, m = line.split(",")[:2]
                    self.util.append(float(u))
                    self.mem.append(float(m))
                except ValueError:
                    pass
            os.unlink(self.path)

    def mean(self):
        """Mean utilization (percent), None without samples."""
        return statistics.mean(self.util) if self.util else None

    def peak_mem_mib(self):
        """Largest device memory in use (MiB), None without samples."""
        return max(self.mem) if self.mem else None


def aggregate_replicas(ms, units, world_size, device="cpu"):
    """Replicas: the job time is the slowest rank's, the work is every rank's.
    Returns (max ms over ranks, sum of units over ranks); one process = as is."""
    if world_size <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t.item()), float(u.item())


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2306_10652_gb300 import lbmfug

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    d, case = load_case(args.nc)
    nx, ny = d["nx"], d["ny"]
    nc = case["nc"]
    prec = {"fp64": lbmfug.LBM_FP64, "fp32dev": lbmfug.LBM_FP32DEV, "fp32": lbmfug.LBM_FP32}[args.precision]
    if args.grid:
        nx, ny = (int(v) for v in args.grid.lower().split("x"))
    sched = {"auto": lbmfug.LBM_SCHED_AUTO, "threepass": lbmfug.LBM_SCHED_THREEPASS,
             "fused": lbmfug.LBM_SCHED_FUSED}[args.schedule]
    rho = initial_density(d, case, nx, ny)
    stream = torch.cuda.Stream()
    kw = dict(precision=prec, schedule=sched, kappa_ref=case["kappa_ref"], stream=stream.cuda_stream,
              monitor_every=1)
    prob = lbmfug.Problem(0, nx, ny, 1, case["a"], case["b"], case["omega"],
                          np.asarray(case["kij"]), case["T"], case["tau"], **kw)
    d_rho = torch.from_numpy(rho.reshape(-1)).to(f"cuda:{local}")
    prob.init_fields_device(d_rho)
    del d_rho
    prob.step(args.warmup)
    prob.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = prob.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    prob.timing_enable(True)  # an event pair around every kernel launch, on the launching stream
    with ClockSampler(local) as clk:
        e0.record(stream)
        prob.step(args.steps)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    launches = prob.launch_count() - l0
    ms = e0.elapsed_time(e1)
    kernels = prob.timing_read()
    prob.timing_enable(False)
    mass, at, nonfinite = prob.monitor()
    N = nx * ny
    ms, node_steps = aggregate_replicas(ms, N * args.steps, ws, device=f"cuda:{local}")
    prob.close()
    value = nc * node_steps / (ms * 1e-3) / 1e9
    spop = 8 if prec == lbmfug.LBM_FP64 else 4
    alg_bytes_per_launch = 2 * 9 * nc * spop * N
    step_ms = ms / args.steps
    pk, pk_kind = peaks()
    step_achieved = alg_bytes_per_launch / (step_ms * 1e-3) / 1e9  # GB/s, whole step
    # The roofline kernel is the fused step kernel: it moves the populations, so it carries the
    # step's algorithmic bytes; the other kernels of the step are listed with their shares.
    kt_total = sum(v[1] for v in kernels.values())
    kernel_table = {n: {"launches": v[0], "ms_per_launch": v[1] / max(v[0], 1),
                        "share": v[1] / kt_total if kt_total > 0 else None} for n, v in kernels.items()}
    step_kernel = next((n for n in kernels if n.startswith("k_fused32")), None)
    dominant = max(kernels, key=lambda n: kernels[n][1]) if kernels else None
    kernel_ms = kernel_table[step_kernel]["ms_per_launch"] if step_kernel else step_ms
    achieved = alg_bytes_per_launch / (kernel_ms * 1e-3) / 1e9  # GB/s, step kernel per launch
    e2e = run_e2e(args, lbmfug, case, rho, nx, ny, prec, sched, local) \
        if (rank == 0 and not args.no_e2e) else None
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None
    cpu = cpu_baseline(case, nx, ny, rho) if (ws == 1 and not args.no_cpu_baseline) else None
    batched = run_batched(args, lbmfug, local) if not args.no_batched else None
    served = run_served(args, lbmfug) if not args.no_served else None
    served_scale = run_served_scale(args, lbmfug) if not (args.no_served or args.no_serve_scale) else None
    forms = None
    if not args.no_forms:
        forms = {}
        for name, pr, sc, k in (("fp32dev_fused", lbmfug.LBM_FP32DEV, lbmfug.LBM_SCHED_AUTO, 10),
                                ("fp32_fused", lbmfug.LBM_FP32, lbmfug.LBM_SCHED_AUTO, 10),
                                ("fp64_fused", lbmfug.LBM_FP64, lbmfug.LBM_SCHED_AUTO, 4),
                                ("fp64_threepass", lbmfug.LBM_FP64, lbmfug.LBM_SCHED_THREEPASS, 4)):
            if pr == prec and sc == sched:
                continue
            forms[name] = time_form(lbmfug, case, rho, nx, ny, pr, sc, k, 2, local)
        # D3Q19 (no single-pass kernel): the multi-pass LBM_FP32DEV schedule and binary64
        forms["d3q19_fp32dev_multipass"] = time_form_3d(lbmfug, case, 128, lbmfug.LBM_FP32DEV,
                                                        lbmfug.LBM_SCHED_AUTO, 10, 3, local)
        forms["d3q19_fp64_threepass"] = time_form_3d(lbmfug, case, 128, lbmfug.LBM_FP64,
                                                     lbmfug.LBM_SCHED_AUTO, 2, 1, local)
    clocks = clk.summary()
    traffic = traffic_per_launch(args, nc, N)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == lbmfug.LBM_FP64 else "f32",
        "data": "synthetic (seeded PR mixture, uniform state in the spinodal region + 1% noise)",
        "config": {"workload": f"spinodal decomposition D2Q9 {nx}x{ny} periodic, Nc={nc}",
                   "lattice": "D2Q9", "nx": nx, "ny": ny, "nc": nc,
                   "precision": args.precision, "schedule": args.schedule,
                   "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (populations %.2f GB per buffer)" % (9 * nc * spop * N / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic[0],
                     "traffic_kernel": traffic[1],
                     "peak_kind": pk_kind, "algorithmic_bytes_per_node_step": 2 * 9 * nc * spop,
                     "kernel": step_kernel or "step",
                     "kernel_ms_per_launch": kernel_ms,
                     "dominant_kernel": dominant,
                     "kernels": kernel_table,
                     "step": {"achieved": step_achieved, "frac": step_achieved / pk["hbm_gbs"],
                              "note": "the step's algorithmic bytes over the whole step time (all its kernels)"}},
        "forms": forms,
        "batched": batched,
        "served": served,
        "served_at_scale": served_scale,
        "gpu_launches": launches,
        "mass_monitor": {"at_step": at, "nonfinite": nonfinite,
                         "mass": None if mass is None else [float(v) for v in mass]},
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
    }
    if ws > 1:
        dist.destroy_process_group()
    return line


def time_form(lbmfug, case, rho, nx, ny, prec, sched, steps, warmup, local):
    """Nc-GLUPS of one precision/schedule form on the same workload (CUDA events)."""
    import torch
    stream = torch.cuda.Stream()
    prob = lbmfug.Problem(0, nx, ny, 1, case["a"], case["b"], case["omega"], np.asarray(case["kij"]),
                          case["T"], case["tau"], precision=prec, schedule=sched,
                          kappa_ref=case["kappa_ref"], stream=stream.cuda_stream, monitor_every=1)
    d_rho = torch.from_numpy(rho.reshape(-1)).to(f"cuda:{local}")
    prob.init_fields_device(d_rho)
    del d_rho
    prob.step(warmup)
    prob.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    prob.step(steps)
    e1.record(stream)
    e1.synchronize()
    prob.close()
    ms = e0.elapsed_time(e1)
    return {"value": case["nc"] * nx * ny * steps / (ms * 1e-3) / 1e9, "ms_per_step": ms / steps}


def time_form_3d(lbmfug, case, n, prec, sched, steps, warmup, local):
    """Nc-GLUPS and HBM fraction of one form on a D3Q19 n^3 box of the same
    mixture (uniform composition, +-1 % seeded noise), CUDA events."""
    import torch
    from paper_2306_10652_gb300 import synth
    nc = case["nc"]
    z = np.asarray(case["z"])
    rho = (z[:, None, None, None] * case["rho_molar_total"]) * synth.multiplicative_noise(12, (nc, n, n, n), 0.01)
    stream = torch.cuda.Stream()
    prob = lbmfug.Problem(1, n, n, n, case["a"], case["b"], case["omega"], np.asarray(case["kij"]),
                          case["T"], case["tau"], precision=prec, schedule=sched, kappa_ref=case["kappa_ref"],
                          stream=stream.cuda_stream)
    d_rho = torch.from_numpy(rho.reshape(-1)).to(f"cuda:{local}")
    prob.init_fields_device(d_rho)
    del d_rho
    prob.step(warmup)
    prob.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    prob.timing_enable(True)
    e0.record(stream)
    prob.step(steps)
    e1.record(stream)
    e1.synchronize()
    kernels = prob.timing_read()
    prob.close()
    ms = e0.elapsed_time(e1) / steps
    N = n ** 3
    spop = 8 if prec == lbmfug.LBM_FP64 else 4
    alg = 2 * 19 * nc * spop * N
    pk, _ = peaks()
    return {"value": nc * N / (ms * 1e-3) / 1e9, "ms_per_step": ms, "box": f"D3Q19 {n}^3",
            "roofline_frac": alg / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
            "algorithmic_bytes_per_node_step": 2 * 19 * nc * spop,
            "kernels_ms_per_launch": {k: v[1] / max(v[0], 1) for k, v in kernels.items()}}


def run_e2e(args, lbmfug, case, rho, nx, ny, prec, sched, local):
    """Same metric through the public C ABI with host buffers: pinned-host
    densities in (H2D inside lbm_init_fields), K steps, densities out (D2H)."""
    import torch
    N = nx * ny
    nc = case["nc"]
    h_in = torch.empty(nc * N, dtype=torch.float64, pin_memory=True).numpy()
    h_in[:] = rho.reshape(-1)
    h_out = torch.empty(nc * N, dtype=torch.float64, pin_memory=True).numpy()
    prob = lbmfug.Problem(0, nx, ny, 1, case["a"], case["b"], case["omega"], np.asarray(case["kij"]),
                          case["T"], case["tau"], precision=prec, schedule=sched,
                          kappa_ref=case["kappa_ref"], monitor_every=1)
    prob.init_fields(h_in)          # first call allocates; not timed
    prob.step(args.warmup)          # warm-up, as in the device-timed leg (the first step of a size also
    prob.synchronize()              # times the candidate launch geometries, once per process)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob.init_fields(h_in)
    prob.step(args.e2e_steps)
    prob.moments(("rho",), out_arrays={"rho": h_out})
    t1 = time.perf_counter()
    prob.close()
    wall = t1 - t0
    return {"value": nc * N * args.e2e_steps / wall / 1e9, "unit": METRIC, "steps": args.e2e_steps,
            "h2d_bytes_per_step": nc * N * 8 / args.e2e_steps, "d2h_bytes_per_step": nc * N * 8 / args.e2e_steps,
            "wall_s": wall}


def cpu_info():
    """(logical cores, CPU model) of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_rate(case, rho, crop, steps, threads):
    """Nc*GLUPS of the CPU oracle on a crop x crop piece of the workload."""
    from oracle import OracleProblem
    from oracle.orc import set_threads
    nc = case["nc"]
    used = set_threads(threads)
    P = OracleProblem(0, crop, crop, 1, case["a"], case["b"], case["omega"], np.asarray(case["kij"]),
                      T=case["T"], tau=case["tau"], kappa_ref=case["kappa_ref"])
    g = P.init_equilibrium(np.ascontiguousarray(rho[:nc, :, :crop, :crop]))
    t0 = time.perf_counter()
    P.step(g, steps)
    dt = time.perf_counter() - t0
    return nc * crop * crop * steps / dt / 1e9, dt, used


def config0_rate():
    """The binary flat-interface configuration in full (D2Q9 128 x 4, Nc = 2,
    binary64, tau = 1, 5000 steps) on the oracle: Nc*GLUPS, seconds."""
    from oracle.orc import set_threads
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import oracle_problem, seeded_mixture
    from oracle.workloads import slab, two_phase_pressure
    from paper_2306_10652_gb300 import synth
    nx, ny, nc = 128, 4, 2
    c = seeded_mixture(0, nc, 0, (1, ny, nx))
    orc = oracle_problem(c, 0, (1, ny, nx))
    _, fl = two_phase_pressure(orc, np.ones(nc) / nc, 0.5)
    rho = np.repeat(slab(fl.rhoi_V, fl.rhoi_L, nx)[:, None, None, :], ny, axis=2)
    rho = rho * synth.multiplicative_noise(0, rho.shape, 1e-3)
    set_threads(1)  # 512 nodes: below the oracle's parallel threshold
    g = orc.init_equilibrium(rho)
    t0 = time.perf_counter()
    orc.step(g, 5000)
    dt = time.perf_counter() - t0
    return nc * nx * ny * 5000 / dt / 1e9, dt


def cpu_baseline(case, nx, ny, rho, crop=256):
    """The oracle on the host cores (a reported baseline, not the target):
    the workload on a 256 x 256 crop single-threaded and on every core, the
    same crop for Nc = 1..10, and the binary flat-interface configuration in
    full.  About 20-30 s of CPU work."""
    ncores, model = cpu_info()
    v1, dt1, _ = oracle_rate(case, rho, crop, 1, 1)
    vN, dtN, used = oracle_rate(case, rho, crop, 2, 0)
    per_nc = {}
    d = json.load(open(WORKLOAD_FILE))
    for nc in range(1, 11):
        cs = [c for c in d["cases"] if c["nc"] == nc][0]
        r = initial_density(d, cs, crop, crop)
        a, _, _ = oracle_rate(cs, r, crop, 1, 1)
        b, _, _ = oracle_rate(cs, r, crop, 2, 0)
        per_nc[nc] = {"single_thread": a * 1e3, "all_cores": b * 1e3}
    c0, dt0 = config0_rate()
    from oracle.orc import set_threads
    set_threads(0)
    return {"value": vN, "unit": METRIC, "cores": used, "kind": "oracle",
            "sample": f"{crop}x{crop} crop of the workload, 2 steps on {used} threads ({dtN:.1f} s)",
            "single_thread": {"value": v1, "sample": f"same crop, 1 step ({dt1:.1f} s)"},
            "host": {"nproc": ncores, "cpu_model": model},
            "per_nc_mlups_256crop": per_nc,
            "config0_full": {"value_nc_mlups": c0 * 1e3, "seconds": dt0,
                             "workload": "binary flat interface D2Q9 128x4, Nc=2, 5000 steps, one thread"}}


TERNARY_FILE = os.path.join(ROOT, "paper_2306_10652_gb300", "workloads", "ternary_sweep.json")


def ternary_jobs(limit=None):
    """The batched sweep's slabs: Eq. (15) profiles at the stored flash densities."""
    d = json.load(open(TERNARY_FILE))
    jobs = []
    for jb in d["jobs"][:limit]:
        nx, ny, SV, W = jb["nx"], jb["ny"], jb["S_V"], d["W"]
        x = np.arange(nx, dtype=float)
        rv = np.asarray(jb["rhoi_V"])[:, None]
        rl = np.asarray(jb["rhoi_L"])[:, None]
        prof = rv + 0.5 * (rl - rv) * (np.tanh(2 * (x - 0.5 * SV * nx) / W)
                                       - np.tanh(2 * (x - (1 - 0.5 * SV) * nx) / W))
        jobs.append((jb["T"], np.repeat(prof[:, None, :], ny, axis=1)))
    return d, jobs


def ulp32(x):
    """Spacing of binary32 numbers at x > 0."""
    return 2.0 ** (np.floor(np.log2(np.float32(x))) - 23)


def tie_line_errors(d, jobs, states, sample):
    """Largest relative deviation of each sampled converged slab's vapour and
    liquid mole fractions (x = 0 and x = nx/2) from the flash compositions
    stored with the slab (the flash at its initial T, p and z, written by
    oracle/make_workloads.py).  The slab's pressure settles slightly away from
    the initial one, so this includes that drift; the tests compare with the
    flash at the slab's own pressure."""
    errs = []
    for k in sample:
        st = states[k]
        if not st["converged"]:
            continue
        rm = st["rho"][:, 0]
        nx = rm.shape[1]
        rV, rL = rm[:, 0], rm[:, nx // 2]
        job = d["jobs"][k]
        y, x = np.asarray(job["y"]), np.asarray(job["x"])
        errs.append(max(np.abs((rV / rV.sum()) / y - 1).max(), np.abs((rL / rL.sum()) / x - 1).max()))
    return errs


def fp64_one_at_a_time(lbmfug, d, jobs, order, tol, every, cap, budget_s):
    """The plain binary64 per-problem path, one slab after the other, each run
    to the same criterion as the batched form (largest density change per
    `every` steps below max(tol, 8 ulp of binary32 at its largest density)),
    until budget_s has passed.  Returns (solves, seconds, node-steps)."""
    t0 = time.perf_counter()
    solved, node_steps = 0, 0
    for k in order:
        if time.perf_counter() - t0 > budget_s:
            break
        T, rho = jobs[k]
        bar = max(tol, 8 * ulp32(1.05 * rho.sum(axis=0).max()))
        p = lbmfug.Problem(0, rho.shape[2], rho.shape[1], 1, d["a"], d["b"], d["omega"], np.asarray(d["kij"]),
                           T, d["tau"], precision=lbmfug.LBM_FP64, kappa_ref=d["kappa_ref"])
        p.init_fields(rho[:, None])
        p.convergence()
        steps = 0
        while steps < cap:
            p.step(every)
            steps += every
            if p.convergence() < bar:
                solved += 1
                break
        node_steps += steps * rho.shape[1] * rho.shape[2]
        p.close()
    return solved, time.perf_counter() - t0, node_steps


def run_batched(args, lbmfug, local):
    """Batched form: all sweep slabs to convergence (solves/s) with the tie-line
    error of a sample against the oracle flash, and the plain binary64
    per-problem path measured on a sample of the same slabs to the same
    criterion."""
    d, jobs = ternary_jobs(args.batch_jobs)
    tol, every, cap = 2e-6, 1000, args.batch_max_steps
    t0 = time.perf_counter()
    with lbmfug.Batch(d["a"], d["b"], d["omega"], np.asarray(d["kij"]), d["tau"], jobs,
                      precision=lbmfug.LBM_FP32, kappa_ref=d["kappa_ref"]) as bt:
        t1 = time.perf_counter()
        bt.run(cap, every, tol)
        t2 = time.perf_counter()
        states = [bt.state(k) for k in range(len(jobs))]
        info = bt.info()
    conv = sum(s["converged"] for s in states)
    failed = sum(s["failed"] for s in states)
    node_steps = sum(s["steps"] * r.shape[1] * r.shape[2] for s, (_, r) in zip(states, jobs))
    wall = t2 - t1
    rng = np.random.default_rng(5)
    sample = rng.permutation(len(jobs))
    errs = tie_line_errors(d, jobs, states, sample[:48])
    # the binary64 path on slabs the batched form solved, in the same seeded order
    solved = [k for k in sample if states[k]["converged"]]
    s64, w64, ns64 = fp64_one_at_a_time(lbmfug, d, jobs, solved, tol, every, cap, args.batch_fp64_s)
    unconv = [k for k, s in enumerate(states) if not s["converged"] and not s["failed"]]
    return {"jobs": len(jobs), "converged": conv, "failed": failed,
            "criterion": f"max|drho| per {every} steps < max({tol}, 8 ulp_binary32(largest total density))",
            "max_steps": cap, "wall_s": wall, "setup_s": t1 - t0, "solves_per_s": conv / wall,
            "node_steps_per_s": node_steps / wall, "threads": info["threads"], "ctas": info["ctas"],
            "rounds": info["rounds"], "precision": "fp32 (binary32 state and thermodynamics)",
            "unconverged_last_drho": sorted(float(states[k]["last_drho"]) for k in unconv)[-5:],
            "tie_line_vs_flash": {"slabs": len(errs), "max_rel": float(max(errs)) if errs else None,
                                  "median_rel": float(np.median(errs)) if errs else None,
                                  "against": "the stored flash at each slab's initial (T, p, z)"},
            "fp64_one_at_a_time": {"measured": True, "solves": s64, "wall_s": w64,
                                   "solves_per_s": s64 / w64 if w64 > 0 else None,
                                   "node_steps_per_s": ns64 / w64 if w64 > 0 else None,
                                   "sample": "slabs the batched form converged, in a seeded random order, "
                                             "each alone to the same criterion"}}


SERVE_FILE = os.path.join(ROOT, "paper_2306_10652_gb300", "workloads", "served_requests.json")


def served_field(r, W):
    """Initial densities of one request: Eq. (15) slab along x (D2Q9 or a D3Q19
    box), or Eq. (13) droplet with the liquid area fraction 1 - S_V."""
    nx, ny, nz, SV = r["nx"], r["ny"], r["nz"], r["S_V"]
    rv = np.asarray(r["rhoi_V"])[:, None, None, None]
    rl = np.asarray(r["rhoi_L"])[:, None, None, None]
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float), np.arange(nx, dtype=float),
                          indexing="ij")
    if r["kind"] == "droplet":
        R = np.sqrt((1.0 - SV) * nx * ny / np.pi)
        dist = np.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2) - R
        return 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2 * dist / W)
    return rv + 0.5 * (rl - rv) * (np.tanh(2 * (x - 0.5 * SV * nx) / W) - np.tanh(2 * (x - (1 - 0.5 * SV) * nx) / W))


def run_served(args, lbmfug):
    """Served form: the requests arrive with their Poisson gaps and run to
    convergence under the 80 % memory budget; latency percentiles and solves/s
    count converged requests only.  The plain binary64 path is measured on the
    same requests one at a time, each to the same criterion, for a bounded
    time."""
    d = json.load(open(SERVE_FILE))
    reqs = d["requests"]
    tol, every, cap = 2e-6, 1000, args.serve_max_steps
    fields = [served_field(r, d["W"]) for r in reqs]
    with lbmfug.Server(0.8, max_active=args.serve_slots) as srv, BusySampler(0) as busy:
        t0 = time.perf_counter()
        ids = []
        for r, rho in zip(reqs, fields):
            time.sleep(r["arrival_gap_s"] / args.serve_rate)
            ids.append(srv.submit(r["lattice"], r["a"], r["b"], r["omega"], np.asarray(r["kij"]), r["T"], d["tau"],
                                  rho, precision=lbmfug.LBM_FP32DEV, check_every=every, max_steps=cap, tol=tol,
                                  kappa_ref=d["kappa_ref"]))
        srv.wait_all()
        t1 = time.perf_counter()
        polls = [srv.poll(j) for j in ids]
        stats = srv.stats()
    busy_pct = busy.mean()
    conv = [p for p in polls if p["state"] == "converged"]
    lat = np.array([p["latency_s"] for p in conv]) if conv else np.array([np.nan])
    work = sum(p["steps"] * r["nc"] * r["nx"] * r["ny"] * r["nz"] for p, r in zip(polls, reqs))
    # binary64, one request at a time, each to the same criterion, for a bounded time
    order = np.random.default_rng(6).permutation(len(reqs))
    b0 = time.perf_counter()
    solved64 = 0
    for k in order:
        if time.perf_counter() - b0 > args.serve_fp64_s:
            break
        r, rho = reqs[k], fields[k]
        bar = max(tol, 8 * ulp32(1.05 * rho.sum(axis=0).max()))
        prob = lbmfug.Problem(r["lattice"], r["nx"], r["ny"], r["nz"], r["a"], r["b"], r["omega"],
                              np.asarray(r["kij"]), r["T"], d["tau"], precision=lbmfug.LBM_FP64,
                              kappa_ref=d["kappa_ref"])
        prob.init_fields(rho)
        prob.convergence()
        steps = 0
        while steps < cap:
            prob.step(every)
            steps += every
            if prob.convergence() < bar:
                solved64 += 1
                break
        prob.close()
    w64 = time.perf_counter() - b0
    return {"requests": len(reqs), "converged": len(conv),
            "exhausted": sum(p["state"] == "exhausted" for p in polls),
            "failed": sum(p["state"] == "failed" for p in polls),
            "criterion": f"max|drho| per {every} steps < max({tol}, 8 ulp_binary32(1.05 x largest total density)), "
                         f"cap {cap} steps",
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "latency_over": "converged requests",
            "wall_s": t1 - t0, "solves_per_s": len(conv) / (t1 - t0),
            "arrival_rate_per_s": args.serve_rate / float(np.mean([r["arrival_gap_s"] for r in reqs])),
            "gpu_busy_pct": busy_pct,
            "nc_node_steps_per_s": work / (t1 - t0), "slots": args.serve_slots,
            "peak_bytes": stats["peak_bytes"], "budget_bytes": stats["budget_bytes"], "rounds": stats["rounds"],
            "precision": "fp32dev (binary32 populations; thermodynamics double-binary32: fused D2Q9, "
                         "multi-pass D3Q19)",
            "fp64_one_at_a_time": {"measured": True, "solves": solved64, "wall_s": w64,
                                   "solves_per_s": solved64 / w64 if w64 > 0 else None,
                                   "sample": "requests in a seeded random order, each alone to the criterion"}}


def scale_field(r, n_x, shape, W):
    """Eq. (15) slab along x of one request at another size: the profile
    along x broadcast over y and z (molar densities [Nc][nz][ny][nx])."""
    SV = r["S_V"]
    rv = np.asarray(r["rhoi_V"])[:, None]
    rl = np.asarray(r["rhoi_L"])[:, None]
    x = np.arange(n_x, dtype=float)[None, :]
    prof = rv + 0.5 * (rl - rv) * (np.tanh(2 * (x - 0.5 * SV * n_x) / W) - np.tanh(2 * (x - (1 - 0.5 * SV) * n_x) / W))
    return np.ascontiguousarray(np.broadcast_to(prof[:, None, None, :], (prof.shape[0],) + tuple(shape)))


def run_served_scale(args, lbmfug):
    """The served form at the largest geometries of the served configuration:
    D3Q19 slab boxes of 160^3-192^3 and D2Q9 slabs of 1024^2, with the
    mixtures of the served request set (Nc 2..10), every request run for a
    fixed number of steps (boxes this size relax over millions of steps, so
    they are not run to convergence).  All are submitted at once, so the 80 %
    memory budget, not the slot count, decides how many run together."""
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    d = json.load(open(SERVE_FILE))
    r3 = [r for r in d["requests"] if r["lattice"] == 1]
    r2 = [r for r in d["requests"] if r["lattice"] == 0]
    plan = [(1, r, (n, n, n)) for n in (192, 192, 176, 176, 160, 160) for r in r3]
    plan += [(0, r, (1, 1024, 1024)) for r in r2[:args.scale_2d]]
    steps, every = args.scale_steps, max(1, args.scale_steps // 2)
    est = [lbmfug.lbm_server_estimate_bytes(lat, sh[2], sh[1], sh[0], r["nc"], lbmfug.LBM_FP32DEV)
           for lat, r, sh in plan]
    with lbmfug.Server(0.8, max_active=len(plan)) as srv, BusySampler(0) as busy:
        t0 = time.perf_counter()
        ids = []
        for lat, r, sh in plan:
            rho = scale_field(r, sh[2], sh, d["W"])
            ids.append(srv.submit(lat, r["a"], r["b"], r["omega"], np.asarray(r["kij"]), r["T"], d["tau"], rho,
                                  precision=lbmfug.LBM_FP32DEV, check_every=every, max_steps=steps, tol=0.0,
                                  kappa_ref=d["kappa_ref"]))
            del rho
        t_sub = time.perf_counter() - t0
        srv.wait_all()
        t1 = time.perf_counter()
        polls = [srv.poll(j) for j in ids]
        times = [srv.times(j) for j in ids]
        stats = srv.stats()
        adm = srv.admission()
    work = sum(p["steps"] * r["nc"] * sh[0] * sh[1] * sh[2] for p, (lat, r, sh) in zip(polls, plan))
    q = np.array([t[0] for t in times])
    run = np.array([t[1] for t in times])
    return {"requests": len(plan),
            "geometries": f"{len([1 for p in plan if p[0] == 1])} D3Q19 boxes 160^3-192^3, "
                          f"{len([1 for p in plan if p[0] == 0])} D2Q9 1024^2; Nc of the served mixtures",
            "steps_per_request": steps, "finished": sum(p["state"] == "exhausted" for p in polls),
            "failed": sum(p["state"] == "failed" for p in polls),
            "estimated_bytes_all": float(sum(est)), "budget_bytes": stats["budget_bytes"],
            "peak_bytes": stats["peak_bytes"], "peak_active": adm["peak_active"],
            "memory_waits": adm["memory_waits"], "device_mem_peak_mib": busy.peak_mem_mib(),
            "wall_s": t1 - t0, "submit_s": t_sub, "nc_node_steps_per_s": work / (t1 - t0),
            "queued_s": {"p50": float(np.percentile(q, 50)), "max": float(q.max())},
            "run_s": {"p50": float(np.percentile(run, 50)), "max": float(run.max())},
            "gpu_busy_pct": busy.mean(),
            "precision": "fp32dev (multi-pass D3Q19, fused D2Q9)"}


def run_reference(args):
    """The oracle as the reference arm: each bench step a bounded sample of the
    workload (a 256 x 256 crop, all host cores), on rank 0 only."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return None
    d, case = load_case(args.nc)
    nx, ny = d["nx"], d["ny"]
    crop = 256
    rho = initial_density(d, case, crop, crop)
    ncores, model = cpu_info()
    for _ in range(args.warmup):
        oracle_rate(case, rho, crop, 1, 0)
    _, dt1, used = oracle_rate(case, rho, crop, 1, 0)
    per_step_s = max(0.1, 60.0 / max(args.steps, 1))
    inner = max(1, int(per_step_s / max(dt1, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(case, rho, crop, inner, 0)
    wall = time.perf_counter() - t0
    nc = case["nc"]
    value = nc * crop * crop * inner * args.steps / wall / 1e9
    sample = f"{crop}x{crop} crop of the workload, {inner} oracle steps per bench step, {used} threads"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"spinodal decomposition D2Q9 {nx}x{ny} periodic, Nc={nc}",
                                            "lattice": "D2Q9", "nx": nx, "ny": ny, "nc": nc},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": used, "kind": "oracle", "sample": sample,
                             "host": {"nproc": ncores, "cpu_model": model}},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--nc", type=int, default=10)
    ap.add_argument("--precision", default="fp32dev", choices=["fp32dev", "fp32", "fp64"])
    ap.add_argument("--no-forms", action="store_true", help="skip the comparison forms")
    ap.add_argument("--grid", default=None, help="NXxNY override of the workload grid (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=40, help="steps of the end-to-end job (init from host, steps, "
                                                               "densities to host)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-jobs", type=int, default=None, help="first N jobs of the sweep")
    ap.add_argument("--batch-max-steps", type=int, default=1000000)
    ap.add_argument("--batch-fp64-s", type=float, default=60.0, help="seconds of the binary64 one-at-a-time sample")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-max-steps", type=int, default=200000)
    ap.add_argument("--serve-fp64-s", type=float, default=60.0, help="seconds of the binary64 one-at-a-time sample")
    ap.add_argument("--serve-rate", type=float, default=1.0, help="arrival-rate multiplier of the served requests")
    ap.add_argument("--no-serve-scale", action="store_true", help="skip the served form at the largest geometries")
    ap.add_argument("--scale-steps", type=int, default=200, help="steps per request of the served form at scale")
    ap.add_argument("--scale-2d", type=int, default=8, help="D2Q9 1024^2 requests of the served form at scale")
    ap.add_argument("--schedule", default="auto", choices=["auto", "threepass", "fused"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
