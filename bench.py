"""Benchmark: Taylor-Green vortex at 256^3, nu = 1/1600, FP64, Bogacki-Shampine 5(4) with
embedded-error step control (rtol = atol = 1e-6), through the libdns C ABI.

One "step" is one attempted BS5 step: stage sums, 7 right-hand-side evaluations (the 8th
stage's derivative is carried over, first same as last), the error norm and the controller.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` = right-hand-side evaluations per second over the timed steps
(whole job: summed over ranks); `sim_time_per_gpu_s` = simulated time advanced per second.
`--impl reference` times the FP64 CPU oracle on the same workload (each step one oracle
right-hand-side evaluation of the same 256^3 field: a bounded sample).  Multi-GPU runs are
independent replicas (the method has no exchange step on one field per GPU here).
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Derived peak of the double-word form (bench --precision fp32x2): FP32 instruction rate
# 152 SMs x 128 lanes x 2.07 GHz = 40.3e12/s; a butterfly sum costs 8 FP32 instructions (plus
# 3 per stored value to renormalise), a complex product 38 (6 flops): a radix-2 butterfly with
# its twiddle (10 flops) costs 38 + 4 x 8 + 2 x 3 = 76, i.e. 7.6 FP32 instructions per nominal
# FFT flop.
DW_PEAK_TFLOPS = 40.3 / 7.6
METRIC = "sim-time/GPU-s at fixed L2 error vs FP64 oracle; RHS evals/s; % HBM roofline"
UNIT = "RHS evals/s"
N_GRID = 256
NU = 1.0 / 1600.0
TOL = 1e-6
H0 = 0.01
T_END = 2.0
WORKLOAD = "taylor_green_3d_256^3_nu1/1600_bs5_adaptive_tol1e-6_to_t2"
# other workloads of the same path (parity cases; --flow/--grid/--precision select them)
FLOWS = {
    "tg": dict(nu=1.0 / 1600.0, forcing=None),
    "hit": dict(nu=1e-3, forcing=(2.5, None)),
}

# Algorithmic (nominal) FP64 flop counts per launch of each pass, 5 n log2 n per complex
# line of length n, 2.5 n log2 n per real line, plus the pointwise products.
def pass_flops(n):
    import math
    K = (n - 1) // 3
    Mx = My = 2 * K + 1
    Mz = K + 1
    lg = math.log2(n)
    cl = 5 * n * lg          # complex line
    rl = 2.5 * n * lg        # real line
    return {
        "p1_x_inverse_curl": 6 * My * Mz * cl,
        "p2_y_inverse": 6 * n * Mz * cl,
        "p3_z_c2r_cross_r2c": n * n * (9 * rl + 9 * n),
        "p4_y_forward": 3 * n * Mz * cl,
        "p5_x_forward_project": 3 * My * Mz * cl,
    }


def pass_bytes(n, esz=16, ksz=16, ysz=16):
    """Algorithmic HBM bytes per launch (each pass reads its input and writes its output once).
    esz: bytes per complex value of the intermediate fields; ksz: of the output k; ysz: of the
    stage input the x passes read (the fp32 form's step keeps k and the intermediate stage
    inputs in FP32: 8 bytes, and 6 of the 7 stage inputs of an attempt are intermediate)."""
    K = (n - 1) // 3
    M = (2 * K + 1) ** 2 * (K + 1)
    L1 = n * (2 * K + 1) * (K + 1)
    L2 = n * n * (K + 1)
    return {
        "p1_x_inverse_curl": 3 * M * ysz + 6 * L1 * esz,
        "p2_y_inverse": 6 * L1 * esz + 6 * L2 * esz,
        "p3_z_c2r_cross_r2c": 6 * L2 * esz + 3 * L2 * esz,
        "p4_y_forward": 3 * L2 * esz + 3 * L1 * esz,
        "p5_x_forward_project": 3 * L1 * esz + 3 * M * ysz + 3 * M * ksz,
    }


# arithmetic of each form: fp32_mixed transforms in FP32 with FP64 k, stage sums and error
# norm; fp32 also keeps k, the intermediate stage inputs and the increments in FP32
DTYPES = {"fp64": "f64", "fp32_mixed": "f32+f64", "fp32x2": "f32x2+f64", "fp32": "f32+f64state"}

# Nonzero stage coefficients of the Bogacki-Shampine 5(4) pair (Appendix A): terms of the
# stage sums forming the inputs of stages 2..8 (the last one is u_{n+1}), and the terms of
# the embedded error e = h sum_j (b_j - bhat_j) k_j.
BS5_STAGE_TERMS = (1, 2, 3, 4, 5, 6, 6)
BS5_ERR_TERMS = 7


def step_kernel_bytes(n, nc=3, ksz=16):
    """Algorithmic HBM bytes per BS5 attempt of the kernels around the passes: each stage sum
    reads u and its k_j and writes one field; the error norm reads u_n, u_{n+1} and its k_j.
    Fields are the retained box (nc M complex values): the state FP64 (16 bytes); the k_j and
    the intermediate stage inputs ksz bytes per complex value (8 in the fp32 form);
    u_{n+1}, the last stage sum's output, FP64."""
    K = (n - 1) // 3
    cells = nc * (2 * K + 1) ** 2 * (K + 1)
    last = len(BS5_STAGE_TERMS) - 1
    return {"stage_sum": sum(16 + t * ksz + (16 if i == last else ksz)
                             for i, t in enumerate(BS5_STAGE_TERMS)) * cells,
            "err_norm_partials": (2 * 16 + BS5_ERR_TERMS * ksz) * cells}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(items, ws, rank):
    """The units of an ensemble that rank `rank` of `ws` runs: every ws-th, from `rank` on.
    The instances are independent, so the ranks exchange nothing while they run."""
    return list(items)[rank::ws]


def aggregate(dist, ws, ms, n_rhs, sim, device):
    """Whole-job figures over the ranks: the slowest rank's time, the work summed."""
    if ws <= 1:
        return ms, float(n_rhs), sim
    import torch
    t = torch.tensor([ms, float(n_rhs), sim], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item(), sm[2].item()


def host_info():
    """Host cores this process may use, the CPU model, and the memory available (bytes)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            info = fh.read()
        for key in ("model name", "CPU part", "Hardware"):
            for ln in info.splitlines():
                if ln.lower().startswith(key.lower()):
                    model = f"{key}: {ln.split(':', 1)[1].strip()}"
                    break
            if model:
                break
    except Exception:
        pass
    import platform
    mem = None
    try:
        with open("/proc/meminfo") as fh:
            for ln in fh:
                if ln.startswith("MemAvailable:"):
                    mem = int(ln.split()[1]) * 1024
    except Exception:
        pass
    return {"nproc": cores, "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine(), "mem_available_bytes": mem}


# Peak resident memory of one oracle right-hand side at 256^3 (measured: about 5.6 GB; the
# transforms keep a few full-size complex temporaries), scaled by the grid volume.
def oracle_rhs_bytes(n):
    return 6.5e9 * (n / 256.0) ** 3 + 0.3e9


def cpu_workers(n_jobs, n):
    """Worker processes for the oracle baseline: one per host core, as many as the jobs, and
    no more than 60% of the available memory holds."""
    h = host_info()
    w = min(h["nproc"], max(1, n_jobs))
    if h["mem_available_bytes"]:
        w = min(w, max(1, int(0.6 * h["mem_available_bytes"] // oracle_rhs_bytes(n))))
    return w


def _oracle_rhs_job(job):
    """One worker's share: `reps` oracle right-hand sides of the n^3 Taylor-Green field
    (FP64 numpy, one thread).  Returns (reps, start, end) on the monotonic clock, which all
    processes of the host share."""
    n, nu, reps = job
    import synthetic as syn
    from oracle import spectral as sp
    g = sp.Grid(n, n, n)
    uh = g.dealias(syn.taylor_green_3d_hat(n, n, n))
    t0 = time.perf_counter()
    for _ in range(reps):
        sp.rhs(g, uh, nu)
    return reps, t0, time.perf_counter()


def cpu_sample(n_rhs, n_warm=1, n=N_GRID):
    """The oracle timed on the host cores: n_rhs right-hand sides of the n^3 Taylor-Green
    field shared out over single-threaded worker processes (spawned: no state is inherited
    from a process that may hold a CUDA context), after n_warm warm-up evaluations.  Returns
    (right-hand sides per second over the wall time of the timed jobs, that wall time,
    the worker count, host information)."""
    import multiprocessing as mp
    workers = cpu_workers(n_rhs, n)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"                         # one thread per worker: cores = workers
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            if n_warm > 0:
                pool.map(_oracle_rhs_job, [(n, NU, 1)] * min(n_warm, workers), chunksize=1)
            shares = [n_rhs // workers + (1 if i < n_rhs % workers else 0) for i in range(workers)]
            res = pool.map(_oracle_rhs_job, [(n, NU, r) for r in shares if r > 0], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    total = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return total / wall, wall, workers, host_info()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.grid
    v, dt, workers, host = cpu_sample(args.steps, args.warmup, n)
    workload = WORKLOAD if n == N_GRID else f"taylor_green_3d_{n}^3_nu1/1600_bs5_adaptive_tol1e-6"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": workload, "grid": [n] * 3, "nu": NU, "method": "BS5_ADAPTIVE",
                      "rtol": TOL, "atol": TOL},
           "cpu_baseline": {"kind": "oracle", "value": v, "unit": UNIT, "cores": workers,
                            "nproc": host["nproc"], "cpu_model": host["cpu_model"],
                            "machine": host["machine"],
                            "sample": f"{args.steps} oracle right-hand-side evaluations of the "
                                      f"{n}^3 TG field (FP64 numpy with the oracle's own FFT), "
                                      f"shared over {workers} single-threaded worker processes "
                                      f"(one per core, capped by available memory) after "
                                      f"{args.warmup} warm-up evaluations; one BS5 attempt "
                                      "costs 7 of them"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def workload_name(args):
    if args.flow == "tg" and args.grid == N_GRID and args.precision == "fp64":
        base = WORKLOAD
    else:
        nu = FLOWS[args.flow]["nu"]
        base = (f"{'taylor_green_3d' if args.flow == 'tg' else 'hit_forced_k0_4'}_{args.grid}^3_"
                f"nu{nu:g}_bs5_adaptive_tol1e-6_{args.precision}")
    return base if args.mode == "step" else base + "_rhs_only"


def make_field(args):
    import synthetic as syn
    n = args.grid
    if args.flow == "tg":
        return syn.taylor_green_3d_hat(n, n, n)
    return syn.random_solenoidal_hat(n, n, n, seed=1, k0=4.0)


def ensemble_specs(count=64):
    """64 seeded instances: 24 x 64^3, 24 x 96^3, 16 x 128^3; k0 in [2, 6], nu log-uniform in
    [1e-3, 1e-2] (drawn with the SplitMix64 generator of the synthetic inputs, seed = id)."""
    import synthetic as syn
    sizes = [64] * 24 + [96] * 24 + [128] * 16
    out = []
    for i, n in enumerate(sizes[:count]):
        u = syn.uniform01(np.arange(2, dtype=np.uint64), 1000 + i)
        k0 = 2.0 + 4.0 * float(u[0])
        nu = 10.0 ** (-3.0 + float(u[1]))
        out.append((n, k0, nu, i))
    return out


def run_ensemble(args):
    """Config: 64 independent simulations, BS5 adaptive tol 1e-6 each to t_end; one graph
    launch (dns_integrate_batch) against the same instances integrated one after another."""
    import torch
    import torch.distributed as dist

    import synthetic as syn
    from paper_1810_10197_gb300 import Dns, build
    from paper_1810_10197_gb300.dns import DnsBatch
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    all_specs = ensemble_specs(args.count)
    specs = shard(all_specs, ws, rank)      # each rank its own instances (weak scaling)
    t_end = args.t_end
    fields = [syn.random_solenoidal_hat(n, n, n, seed=i, k0=k0) for (n, k0, nu, i) in specs]
    prec = args.precision
    b = DnsBatch([dict(nx=n, nu=nu, precision=prec) for (n, k0, nu, i) in specs])
    tiles = [inst.autotune() for inst in b.instances]
    # warm-up: one short batched integration
    for inst, f in zip(b.instances, fields):
        inst.set_state(torch.from_numpy(f).cuda(), 0.0)
    b.integrate("BS5_ADAPTIVE", [0.01] * len(specs), [TOL] * len(specs), [TOL] * len(specs), [H0] * len(specs))
    for inst, f in zip(b.instances, fields):
        inst.set_state(torch.from_numpy(f).cuda(), 0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = b.integrate("BS5_ADAPTIVE", [t_end] * len(specs), [TOL] * len(specs), [TOL] * len(specs),
                        [H0] * len(specs))
    torch.cuda.synchronize()
    batched_s = time.perf_counter() - t0
    n_rhs = sum(i.n_rhs for i in infos)
    # the same instances, one after another through dns_integrate
    seq_s, seq_rhs = 0.0, 0
    for (n, k0, nu, i), f in zip(specs, fields):
        d = Dns(n, nu=nu, precision=prec)
        d.autotune()
        d.set_state(torch.from_numpy(f).cuda(), 0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = d.integrate(t_end, "BS5_ADAPTIVE", TOL, TOL, h0=H0)
        torch.cuda.synchronize()
        seq_s += time.perf_counter() - t0
        seq_rhs += info.n_rhs
        d.close()
    _, n_rej, _ = aggregate(dist, ws, 0.0, sum(i.n_rej for i in infos), 0.0, "cuda")
    batched_s, n_rhs, _ = aggregate(dist, ws, batched_s, n_rhs, 0.0, "cuda")
    seq_s, seq_rhs, _ = aggregate(dist, ws, seq_s, seq_rhs, 0.0, "cuda")
    if rank != 0:
        b.close()
        dist.destroy_process_group()
        return 0
    sim = len(all_specs) * t_end
    # algorithmic HBM traffic of the batched run: each instance's right-hand sides (five
    # passes) and attempts (stage sums, error norm) at its own grid
    esz = 8 if prec in ("fp32_mixed", "fp32") else 16
    ksz = 8 if prec == "fp32" else 16
    ysz = (6 * 8 + 16) / 7 if prec == "fp32" else 16
    moved = 0.0
    for (n, k0, nu, i), inf in zip(specs, infos):
        moved += inf.n_rhs * sum(pass_bytes(n, esz=esz, ksz=ksz, ysz=ysz).values())
        moved += (inf.n_acc + inf.n_rej) * sum(step_kernel_bytes(n, ksz=ksz).values())
    peaks, peak_src = load_peaks()
    hbm_frac = moved / batched_s / 1e9 / peaks["hbm_gbs"] if ws == 1 else None
    out = {"metric": METRIC, "value": n_rhs / batched_s, "unit": UNIT, "n_gpus": ws, "steps": 1,
           "warmup": 1, "ms_per_step": batched_s * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPES[prec],
           "data": "synthetic",
           "config": {"workload": f"ensemble_{len(all_specs)}x(24x64^3,24x96^3,16x128^3)_bs5_tol1e-6_to_t{t_end:g}",
                      "precision": prec, "tiles": tiles, "parallelism": f"instances sharded over {ws} rank(s)"},
           "sim_time_per_gpu_s": sim / batched_s,
           "sequential": {"rhs_evals_per_s": seq_rhs / seq_s, "sim_time_per_gpu_s": sim / seq_s,
                          "seconds": seq_s},
           "batched_seconds": batched_s, "speedup_vs_sequential": seq_s / batched_s,
           "algorithmic_bytes": moved if ws == 1 else None,
           "hbm_frac_of_measured": hbm_frac,
           "hbm_frac_basis": "algorithmic bytes of every instance's passes and step kernels over "
                             f"the batched wall time, against {peak_src} hbm_gbs",
           "rhs_evals": int(n_rhs), "rejected": int(n_rej)}
    print(json.dumps(out), flush=True)
    b.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def at_error(curve, e, key):
    """log-log interpolation of `key` on an error-versus-cost curve at error e (None outside
    the curve's range)."""
    pts = sorted((c["l2_error"], c[key]) for c in curve if c["l2_error"] > 0)
    for (e0, v0), (e1, v1) in zip(pts, pts[1:]):
        if e0 <= e <= e1:
            w = (math.log(e) - math.log(e0)) / (math.log(e1) - math.log(e0)) if e1 > e0 else 0.0
            return math.exp(math.log(v0) + w * (math.log(v1) - math.log(v0)))
    return None


def run_accuracy(args):
    """Simulated time per GPU-second at a fixed final-state L2 error on the Taylor-Green vortex
    at 256^3, nu = 1/1600, t in [0, T] (or the forced HIT flow with --flow hit).  Error-versus-
    cost curves (Section 3's comparison) for BS5 adaptive over tolerances, RK4 over halving
    steps, DP5, the FP32-mixed, fp32 and double-word forms, all against a time-converged FP64
    reference (BS5 at tol 1e-10); comparisons at equal error interpolate each curve in log-log.
    Energy and enstrophy are traced every step."""
    import torch

    from paper_1810_10197_gb300 import Dns, build
    torch.cuda.set_device(0)
    build.build()
    n, T = args.grid, args.t_end
    nu = FLOWS[args.flow]["nu"]
    u0 = make_field(args)
    u0_dev = torch.from_numpy(u0).cuda()
    forcing = None
    if args.flow == "hit":
        d0 = Dns(n, nu=nu)
        d0.set_state(u0_dev, 0.0)
        forcing = (FLOWS["hit"]["forcing"][0], d0.diagnostics()[2])
        d0.close()

    def run(method, tol, h0, precision="fp64", trace=False):
        d = Dns(n, nu=nu, precision=precision, forcing=forcing)
        d.autotune()
        d.set_state(u0_dev, 0.0)
        if trace:
            d.set_trace(100000, diagnostics=True)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        info = d.integrate(T, method, tol, tol, h0=h0)
        ev1.record()
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) * 1e-3
        u = d.get_state()
        tr = d.trace() if trace else None
        d.close()
        return u, info, sec, tr

    t_start = time.perf_counter()
    u_ref, i_ref, s_ref, _ = run("BS5_ADAPTIVE", 1e-10, H0)
    nrm = np.linalg.norm(u_ref)

    def rec(u, i, sec):
        return {"l2_error": float(np.linalg.norm(u - u_ref) / nrm), "rhs_evals": int(i.n_rhs),
                "accepted": int(i.n_acc), "rejected": int(i.n_rej), "gpu_seconds": sec,
                "sim_time_per_gpu_s": T / sec}

    curves = {"bs5_fp64": [], "rk4_fp64": [], "dp5_fp64": [], "bs5_fp32mixed": [], "bs5_fp32": [],
              "bs5_fp32x2": []}
    trace = None
    for tol in args.tols:
        u, i, sec, tr = run("BS5_ADAPTIVE", tol, H0, trace=(tol == TOL))
        curves["bs5_fp64"].append(dict(tol=tol, **rec(u, i, sec)))
        if tol == TOL:
            acc = tr[tr[:, 3] > 0.5]
            trace = {"t": (acc[:, 0] + acc[:, 1]).tolist(), "h": acc[:, 1].tolist(), "E": acc[:, 5].tolist(),
                     "Omega": acc[:, 6].tolist(), "eps": acc[:, 7].tolist()}
    for tol in args.tols[:4]:
        u, i, sec, _ = run("BS5_ADAPTIVE", tol, H0, precision="fp32_mixed")
        curves["bs5_fp32mixed"].append(dict(tol=tol, **rec(u, i, sec)))
        u, i, sec, _ = run("BS5_ADAPTIVE", tol, H0, precision="fp32")
        curves["bs5_fp32"].append(dict(tol=tol, **rec(u, i, sec)))
    for tol in args.tols:
        u, i, sec, _ = run("BS5_ADAPTIVE", tol, H0, precision="fp32x2")
        curves["bs5_fp32x2"].append(dict(tol=tol, **rec(u, i, sec)))
    for tol in args.dp5_tols:
        u, i, sec, _ = run("DP5_ADAPTIVE", tol, H0)
        curves["dp5_fp64"].append(dict(tol=tol, **rec(u, i, sec)))
    dt = args.rk4_dt
    for _ in range(args.rk4_levels):
        u, i, sec, _ = run("RK4", 0.0, dt)
        curves["rk4_fp64"].append(dict(dt=dt, **rec(u, i, sec)))
        dt /= 2

    cmp = []
    for c in curves["bs5_fp64"]:
        e = c["l2_error"]
        rk_rhs = at_error(curves["rk4_fp64"], e, "rhs_evals")
        rk_sim = at_error(curves["rk4_fp64"], e, "sim_time_per_gpu_s")
        cmp.append({"l2_error": e, "bs5_rhs": c["rhs_evals"], "rk4_rhs_at_same_error": rk_rhs,
                    "rhs_ratio_rk4_over_bs5": (rk_rhs / c["rhs_evals"]) if rk_rhs else None,
                    "bs5_sim_time_per_gpu_s": c["sim_time_per_gpu_s"], "rk4_sim_time_per_gpu_s": rk_sim})
    def vs_fp64(curve):
        out = []
        for c in curve:
            e = c["l2_error"]
            fp64_sim = at_error(curves["bs5_fp64"], e, "sim_time_per_gpu_s")
            out.append({"l2_error": e, "fp32_sim_time_per_gpu_s": c["sim_time_per_gpu_s"],
                        "fp64_sim_time_per_gpu_s_at_same_error": fp64_sim,
                        "speedup": (c["sim_time_per_gpu_s"] / fp64_sim) if fp64_sim else None})
        return out
    fp32_vs_fp64 = vs_fp64(curves["bs5_fp32mixed"])
    fp32lean_vs_fp64 = vs_fp64(curves["bs5_fp32"])
    dw_vs_fp64 = []
    for c in curves["bs5_fp32x2"]:
        e = c["l2_error"]
        fp64_sim = at_error(curves["bs5_fp64"], e, "sim_time_per_gpu_s")
        same_tol = [f for f in curves["bs5_fp64"] if f["tol"] == c["tol"]]
        dw_vs_fp64.append({"tol": c["tol"], "l2_error": e, "fp32x2_sim_time_per_gpu_s": c["sim_time_per_gpu_s"],
                           "fp64_sim_time_per_gpu_s_at_same_error": fp64_sim,
                           "speedup": (c["sim_time_per_gpu_s"] / fp64_sim) if fp64_sim else None,
                           "fp64_same_tol": ({"l2_error": same_tol[0]["l2_error"],
                                              "rhs_evals": same_tol[0]["rhs_evals"],
                                              "sim_time_per_gpu_s": same_tol[0]["sim_time_per_gpu_s"]}
                                             if same_tol else None)})
    main = ([c for c in curves["bs5_fp64"] if c["tol"] == TOL] or curves["bs5_fp64"])[0]
    out = {"metric": METRIC, "value": main["sim_time_per_gpu_s"],
           "unit": f"sim-time/GPU-s (BS5 FP64 tol 1e-6, final L2 error {main['l2_error']:.2e})",
           "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{'taylor_green_3d' if args.flow == 'tg' else 'hit_forced'}_{n}^3_nu{nu:g}_t0-{T:g}",
                      "forcing": forcing,
                      "reference": "BS5 adaptive tol 1e-10, FP64", "reference_rhs_evals": int(i_ref.n_rhs),
                      "reference_gpu_seconds": s_ref},
           "curves": curves, "bs5_vs_rk4_at_equal_error": cmp, "fp32mixed_vs_fp64_at_equal_error": fp32_vs_fp64,
           "fp32_vs_fp64_at_equal_error": fp32lean_vs_fp64,
           "fp32x2_vs_fp64_at_equal_error": dw_vs_fp64,
           "trace_bs5_fp64_tol1e-6": trace, "wall_seconds": time.perf_counter() - t_start}
    print(json.dumps(out), flush=True)
    return 0


def run_controllers(args):
    """The learned step-size proposal against the Section 2.2.1 (I) and PI controllers on
    periodic Boussinesq Rayleigh-Taylor (128 x 128 x 256, Atwood 0.5, tanh interfaces of width
    0.05, multimode perturbation 1e-3, nu = kappa = 1e-3, Ri = 1), each over a tolerance
    sweep and compared at equal final error.  The network corrects the PI factor; candidates
    are trained on the GPU from PI-controlled trajectories of Taylor-Green and forced-HIT
    flows (32^3 and 48^3, tolerances 1e-5..1e-8) and small RT runs (16x16x32, seeds 11, 12),
    and the one most efficient at equal error on a validation RT problem (default 64x64x128,
    seed 13, interface width 0.1) is kept (PI itself is a candidate); every run is measured
    against a tol-1e-9 FP64 reference of the same problem."""
    import torch

    import synthetic as syn
    from paper_1810_10197_gb300 import Dns, build, learned
    torch.cuda.set_device(0)
    build.build()
    t_start = time.perf_counter()
    flows = []
    for tol in (1e-5, 1e-6, 1e-7, 1e-8):
        for m, nu in ((32, 0.01), (32, 0.005), (48, 0.003)):
            flows.append(((m, m, m), syn.taylor_green_3d_hat(m, m, m), nu, None, tol, 2.0))
            flows.append(((m, m, m), syn.random_solenoidal_hat(m, m, m, seed=3 + m, k0=3.0), nu, (2.5, 0.05), tol, 1.0))
    X, T = learned.training_set(flows, lambda shape, nu, forcing: Dns(*shape, nu=nu, forcing=forcing),
                                lambda a: torch.from_numpy(a).cuda())
    # small periodic Rayleigh-Taylor runs (seeds 11, 12; neither the validation nor the
    # measured problem) under PI, as in the controller test
    Xr, Tr = [X], [T]
    for seed in (11, 12):
        for tol in (1e-5, 1e-6, 1e-7):
            Ys, Ls = syn.rayleigh_taylor_hat(16, 16, 32, seed=seed, width=0.2, amplitude=1e-2)
            d = Dns(16, 16, 32, nu=1e-3, lengths=Ls, boussinesq=(1e-3, 1.0))
            d.set_controller("PI")
            d.set_state(torch.from_numpy(Ys).cuda(), 0.0)
            d.set_trace(20000)
            d.integrate(3.0, "BS5_ADAPTIVE", tol, tol, h0=1e-3)
            a, b = learned.pairs_from_trace(d.trace())
            Xr.append(a)
            Tr.append(b)
            d.close()
    X, T = np.concatenate(Xr), np.concatenate(Tr)

    vshape = tuple(args.val_shape)

    def run_validation(p, tol):
        # validation problem: the same family as the measured one at a smaller grid and
        # another seed (13), interfaces as wide as the grid resolves, from rest to t_end
        Yv, Lv = syn.rayleigh_taylor_hat(*vshape, seed=13, width=args.val_width)
        d = Dns(*vshape, nu=1e-3, lengths=Lv, boussinesq=(1e-3, 1.0))
        d.set_state(torch.from_numpy(Yv).cuda(), 0.0)
        d.set_controller("PI" if p is None else "MLP", p)
        info = d.integrate(args.t_end, "BS5_ADAPTIVE", tol, tol, h0=1e-3)
        u = d.get_state()
        d.close()
        return u, info.n_rhs

    params, table = learned.select(X, T, run_validation, (1e-5, 1e-6, 1e-7))
    hist = np.zeros(1)
    train_s = time.perf_counter() - t_start
    nx, ny, nz = args.rt_shape
    Y, L = syn.rayleigh_taylor_hat(nx, ny, nz, seed=7)   # set_state keeps the 2/3 box
    Yd = torch.from_numpy(Y).cuda()
    T_end = args.t_end

    def run(kind, tol, precision=args.precision):
        d = Dns(nx, ny, nz, nu=1e-3, lengths=L, boussinesq=(1e-3, 1.0), precision=precision)
        d.autotune()
        d.set_state(Yd, 0.0)
        if kind == "MLP" and params is not None:
            d.set_controller("MLP", params)
        elif kind in ("PI", "MLP"):
            d.set_controller("PI")            # the selection kept the zero network: PI itself
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st, info = d.integrate(T_end, "BS5_ADAPTIVE", tol, tol, h0=1e-3, check=False)
        ev1.record()
        torch.cuda.synchronize()
        u = d.get_state()
        d.close()
        return u, info, ev0.elapsed_time(ev1) * 1e-3, st

    u_ref, i_ref, s_ref, _ = run("I", args.ref_tol, "fp64")
    nrm = np.linalg.norm(u_ref)
    rows = {}
    curves = {"I": [], "PI": [], "MLP": []}
    for kind in ("I", "PI", "MLP"):
        for tol in sorted(set(args.ctrl_tols) | {TOL}, reverse=True):
            u, info, sec, st = run(kind, tol)
            row = {"tol": tol, "status": st, "t": info.t, "rhs_evals": int(info.n_rhs), "accepted": int(info.n_acc),
                   "rejected": int(info.n_rej), "l2_error": float(np.linalg.norm(u - u_ref) / nrm),
                   "gpu_seconds": sec, "sim_time_per_gpu_s": T_end / sec}
            if st == 0:
                curves[kind].append(row)
            if tol == TOL:
                rows[kind] = row
    # each controller against the Section 2.2.1 (I) controller at the same final error
    equal_error = {}
    for kind in ("PI", "MLP"):
        equal_error[kind] = []
        for c in curves[kind]:
            i_rhs = at_error(curves["I"], c["l2_error"], "rhs_evals")
            i_sim = at_error(curves["I"], c["l2_error"], "sim_time_per_gpu_s")
            equal_error[kind].append({"tol": c["tol"], "l2_error": c["l2_error"], "rhs_evals": c["rhs_evals"],
                                      "I_rhs_evals_at_same_error": i_rhs,
                                      "rhs_saving_vs_I": (i_rhs / c["rhs_evals"]) if i_rhs else None,
                                      "sim_time_ratio_vs_I": (c["sim_time_per_gpu_s"] / i_sim) if i_sim else None})
    # the learned correction against its own base, the PI controller, at the same final error
    mlp_vs_pi = []
    for c in curves["MLP"]:
        p_rhs = at_error(curves["PI"], c["l2_error"], "rhs_evals")
        mlp_vs_pi.append({"tol": c["tol"], "l2_error": c["l2_error"], "rhs_evals": c["rhs_evals"],
                          "PI_rhs_evals_at_same_error": p_rhs,
                          "rhs_saving_vs_PI": (p_rhs / c["rhs_evals"]) if p_rhs else None})
    out = {"metric": METRIC, "value": rows["MLP"]["sim_time_per_gpu_s"], "unit": "sim-time/GPU-s (MLP controller)",
           "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True,
           "dtype": DTYPES[args.precision],
           "data": "synthetic",
           "config": {"workload": f"rayleigh_taylor_{nx}x{ny}x{nz}_atwood0.5_t0-{T_end:g}_bs5_tol1e-6",
                      "precision": args.precision,
                      "reference": f"BS5 adaptive tol {args.ref_tol:g} (I controller)",
                      "reference_rhs_evals": int(i_ref.n_rhs), "training_pairs": int(len(X)),
                      "selection": {"validation": f"RT {vshape[0]}x{vshape[1]}x{vshape[2]} seed 13, interface "
                                                  f"width {args.val_width}, t 0-{args.t_end:g}, "
                                                  "tolerances 1e-5..1e-7",
                                    "candidates_efficiency_vs_PI": [list(r) for r in table],
                                    "selected": "zero network (PI)" if params is None else "trained network"},
                      "training_seconds_incl_trajectories_and_selection": train_s},
           "runs": rows,
           "curves": curves,
           "at_equal_error_vs_I": equal_error,
           "mlp_at_equal_error_vs_PI": mlp_vs_pi,
           "mlp_rhs_saving_vs_I": rows["I"]["rhs_evals"] / max(rows["MLP"]["rhs_evals"], 1),
           "wall_seconds": time.perf_counter() - t_start}
    print(json.dumps(out), flush=True)
    return 0


PASS_NAMES = ("p1_x_inverse_curl", "p2_y_inverse", "p3_z_c2r_cross_r2c", "p4_y_forward",
              "p5_x_forward_project")


def fp64_instructions(n, kernel):
    """FP64 thread instructions per launch of a pass at n^3 (ncu, kept in profiles/)."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_instr.json")) as fh:
            return json.load(fh).get(f"fp64_{n}", {}).get(kernel)
    except Exception:
        return None


def analyse(precision, mode, n, prof, n_rhs, attempts, ms, peaks, peak_src, fp64_rate):
    """Roofline of the dominant pass and HBM fractions from per-kernel CUDA-event times.

    prof: {kernel: (launches, total ms)} over the timed region; n_rhs right-hand sides and
    `attempts` step attempts in it (step mode), ms its length.  In step mode every attempt
    also launches the passes for k_1, which return at once when first-same-as-last carries
    k_1 over: a pass does work n_rhs times, not once per launch."""
    fp32 = precision in ("fp32_mixed", "fp32")
    lean = precision == "fp32"
    dwp = precision == "fp32x2"
    flops = pass_flops(n)
    ksz = 8 if (lean and mode == "step") else 16
    ysz = (6 * 8 + 16) / 7 if (lean and mode == "step") else 16
    byts = pass_bytes(n, esz=8 if fp32 else 16, ksz=ksz, ysz=ysz)
    dom = max(PASS_NAMES, key=lambda k: prof.get(k, (0, 0.0))[1])
    nl, tot_ms = prof[dom]
    n_work = n_rhs if mode == "step" else nl
    avg_s = tot_ms * 1e-3 / n_work
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            traffic = json.load(fh).get(f"{precision}_{n}", {}).get(dom)
    except Exception:
        pass
    hbm_gbs = byts[dom] / avg_s / 1e9
    if fp32:
        roof = {"bound": "hbm", "kernel": dom, "achieved": hbm_gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": hbm_gbs / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "flops_achieved_tflops": flops[dom] / avg_s / 1e12}
    elif dwp:
        achieved = flops[dom] / avg_s / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": DW_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / DW_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz = 40.3e12 FP32 "
                               "instructions/s over 7.6 FP32 instructions per nominal FFT flop in "
                               "double-word arithmetic",
                "hbm_achieved_gbs": hbm_gbs, "hbm_frac_of_measured": hbm_gbs / peaks["hbm_gbs"],
                "hbm_peak_source": peak_src}
    else:
        # bound by the FP64 pipe: FP64 instructions per launch (ncu count) over the time,
        # against the pipe's issue rate measured in this run; nominal flops beside it
        nominal = flops[dom] / avg_s / 1e12
        instr = fp64_instructions(n, dom)
        roof = {"bound": "alu", "kernel": dom, "traffic": traffic,
                "hbm_achieved_gbs": hbm_gbs, "hbm_frac_of_measured": hbm_gbs / peaks["hbm_gbs"],
                "hbm_peak_source": peak_src,
                "nominal_flops_tflops": nominal, "nominal_frac_of_1p25_tflops": nominal / 1.25}
        if instr and fp64_rate:
            achieved = instr / avg_s / 1e12
            roof.update({"achieved": achieved, "peak": fp64_rate / 1e12, "unit": "T FP64 instr/s",
                         "frac": achieved / (fp64_rate / 1e12),
                         "fp64_instructions_per_launch": instr,
                         "peak_source": "FP64 pipe issue rate measured in this run "
                                        "(dns_measure_fp64_rate: independent DFMA chains on every SM); "
                                        "instructions per launch from ncu (profiles/fp64_instr.json)"})
        else:
            roof.update({"achieved": nominal, "peak": 1.25, "unit": "TFLOP/s", "frac": nominal / 1.25,
                         "peak_source": "nominal FP64 rate (1.25 TFLOP/s): no measured issue rate "
                                        "or instruction count for this grid"})
    per_kernel = {k: {"launches": v[0], "total_ms": round(v[1], 3), "share": round(v[1] / ms, 4),
                      "avg_ms": round(v[1] / max(v[0], 1), 4)}
                  for k, v in prof.items()}
    rhs_bytes = sum(byts.values())
    moved = {k: byts[k] * n_rhs for k in byts}
    for k, b in step_kernel_bytes(n, ksz=ksz).items():
        moved[k] = b * attempts
    for k, b in moved.items():
        if k in prof and prof[k][1] > 0 and b > 0:
            gbs = b / (prof[k][1] * 1e-3) / 1e9
            per_kernel[k]["hbm_gbs"] = round(gbs, 1)
            per_kernel[k]["hbm_frac_of_measured"] = round(gbs / peaks["hbm_gbs"], 4)
    # per right-hand-side evaluation: the five passes' algorithmic bytes over their time
    pass_ms = sum(prof.get(k, (0, 0.0))[1] for k in PASS_NAMES)
    rhs_frac = rhs_bytes * n_rhs / (pass_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if pass_ms > 0 else None
    step_frac = sum(moved.values()) / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
    return {"roofline": roof, "kernels": per_kernel, "rhs_bytes": rhs_bytes,
            "rhs_hbm_frac_of_measured": rhs_frac, "step_hbm_frac_of_measured": step_frac,
            "rhs_pass_ms": pass_ms / max(n_rhs, 1)}


def timed_attempts(d, stream, steps, warmup, barrier, clocks=None):
    """W untimed then K timed BS5 attempts from the context's state (CUDA events on its
    stream, per-kernel profile).  Returns (ms, profile, info before, info after, clocks)."""
    import torch
    d.enqueue_attempts(warmup, "BS5_ADAPTIVE", TOL, TOL, t_end=T_END, h0=H0)
    i0 = d.info()
    d.profile_enable(True)
    if clocks:
        clocks.start()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    d.enqueue_attempts(steps, "BS5_ADAPTIVE", TOL, TOL, t_end=T_END, h0=0.0)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    i1 = d.info()
    prof = d.profile()
    d.profile_enable(False)
    return ms, prof, i0, i1, clk


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1810_10197_gb300 import Dns, build
    from paper_1810_10197_gb300.dns import dns_measure_fp64_rate

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.Stream()
    n = args.grid
    nu = FLOWS[args.flow]["nu"]
    u0 = make_field(args)
    u0_dev = torch.from_numpy(u0).cuda()
    forcing = None
    if args.flow == "hit":
        # constant power equal to the initial dissipation rate (input recipe)
        d0 = Dns(n, nu=nu, precision="fp64", stream=stream)
        d0.set_state(u0_dev, 0.0)
        _, _, eps0 = d0.diagnostics()
        d0.close()
        forcing = (FLOWS["hit"]["forcing"][0], eps0)
    fp64_rate = None
    if args.precision == "fp64" or args.forms:
        fp64_rate = dns_measure_fp64_rate(stream)[0]

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def make(precision):
        dd = Dns(n, nu=nu, precision=precision, forcing=forcing, stream=stream)
        if args.tiles and precision == args.precision:
            dd.set_tiles(*args.tiles)
            tl = list(args.tiles)
        else:
            tl = dd.autotune()
        dd.set_state(u0_dev, 0.0)
        return dd, tl

    d, tiles = make(args.precision)
    f_dev = torch.empty_like(u0_dev)
    clocks = ClockSampler(local)
    if args.mode == "rhs":
        for _ in range(args.warmup):
            d.rhs(u0_dev, f_dev)
        i0 = d.info()
        d.profile_enable(True)
        clocks.start()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            d.rhs(u0_dev, f_dev)
        ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop()
        i1 = d.info()
        prof = d.profile()
        d.profile_enable(False)
    else:
        ms, prof, i0, i1, clk = timed_attempts(d, stream, args.steps, args.warmup, barrier, clocks)
    n_rhs = (i1.n_rhs - i0.n_rhs) if args.mode == "step" else args.steps
    sim = (i1.t - i0.t) if args.mode == "step" else 0.0
    attempts = (i1.n_acc - i0.n_acc) + (i1.n_rej - i0.n_rej) if args.mode == "step" else 0
    ms_max, n_rhs_tot, sim_tot = aggregate(dist, ws, ms, n_rhs, sim, "cuda")
    value = n_rhs_tot / (ms_max * 1e-3)
    final_state = d.get_state() if (args.forms and args.mode == "step" and ws == 1) else None

    # ---- end to end through the public API with host buffers (pinned) -------------------
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(u0).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        state_bytes = host_in.numel() * host_in.element_size()
        e2e_steps = max(1, min(args.steps, 4))
        if args.mode == "rhs":
            dev_in = torch.empty_like(u0_dev)
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                dev_in.copy_(host_in, non_blocking=True)      # H2D of this step's input
                d.rhs(dev_in, f_dev)
                host_out.copy_(f_dev, non_blocking=True)       # D2H of this step's result
                torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
            e2e_rhs = e2e_steps
            note = "H2D copy from pinned host memory, one dns_rhs, D2H copy of f"
        else:
            d.set_state(host_in, 0.0)
            info = d.step("BS5_ADAPTIVE", H0, TOL, TOL, T_END)
            h = info.h_next
            t_sim = info.t
            d.get_state(host_out)
            barrier()
            t0 = time.perf_counter()
            e2e_rhs = 0
            for _ in range(e2e_steps):
                d.set_state(host_out, t_sim)             # H2D of this step's input
                info = d.step("BS5_ADAPTIVE", h, TOL, TOL, T_END)
                d.get_state(host_out)                    # D2H of this step's result
                e2e_rhs += info.n_rhs
                if info.accepted:
                    t_sim = info.t
                h = info.h_next
            barrier()
            e2e_s = time.perf_counter() - t0
            note = "set_state from pinned host memory, one dns_step, get_state to host"
        h2d = state_bytes
        if args.mode != "rhs":
            # set_state from host memory copies only the retained box (nc M complex128)
            K = (n - 1) // 3
            h2d = host_in.shape[0] * (2 * K + 1) ** 2 * (K + 1) * 16
            note += " (the upload copies only the retained modes)"
        e2e = {"value": e2e_rhs / e2e_s * ws, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": state_bytes, "steps": e2e_steps, "note": note}
    d.close()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    a = analyse(args.precision, args.mode, n, prof, n_rhs, attempts, ms, peaks, peak_src, fp64_rate)

    # ---- the other arithmetic forms on the same field, same step count, same process ------
    forms = None
    if final_state is not None:
        def reference(t):
            # time-converged FP64 state at t: BS5 adaptive, tolerance 1e-10 (Section 3's
            # accuracy reference: the same flow integrated far more accurately)
            r = Dns(n, nu=nu, precision="fp64", forcing=forcing, stream=stream)
            r.set_state(u0_dev, 0.0)
            r.integrate(t, "BS5_ADAPTIVE", 1e-10, 1e-10, h0=H0)
            u = r.get_state()
            r.close()
            return u

        def l2(u, t):
            ref = reference(t)
            return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))

        forms = {"reference": "FP64 BS5 adaptive, tolerance 1e-10, to each run's final time",
                 args.precision: {"value": value, "sim_time_per_gpu_s": sim_tot / (ms_max * 1e-3),
                                  "t_end_state": i1.t, "l2_error_vs_reference": l2(final_state, i1.t),
                                  "rhs_hbm_frac_of_measured": a["rhs_hbm_frac_of_measured"]}}
        for prec in args.forms:
            if prec == args.precision:
                continue
            dd, tl = make(prec)
            fms, fprof, f0, f1, _ = timed_attempts(dd, stream, args.steps, args.warmup, barrier)
            fu = dd.get_state()
            dd.close()
            fr = f1.n_rhs - f0.n_rhs
            fa = analyse(prec, "step", n, fprof, fr, (f1.n_acc - f0.n_acc) + (f1.n_rej - f0.n_rej),
                         fms, peaks, peak_src, fp64_rate)
            forms[prec] = {"value": fr / (fms * 1e-3), "unit": UNIT, "dtype": DTYPES[prec], "tiles": tl,
                           "sim_time_per_gpu_s": (f1.t - f0.t) / (fms * 1e-3),
                           "rhs_evals": fr, "accepted": f1.n_acc - f0.n_acc, "rejected": f1.n_rej - f0.n_rej,
                           "t_end_state": f1.t, "l2_error_vs_reference": l2(fu, f1.t),
                           "rhs_hbm_frac_of_measured": fa["rhs_hbm_frac_of_measured"],
                           "step_hbm_frac_of_measured": fa["step_hbm_frac_of_measured"],
                           "rhs_pass_ms": fa["rhs_pass_ms"], "roofline": fa["roofline"]}

    launches = sum(v[0] for v in prof.values())
    cpu = None
    if ws == 1 and not args.no_cpu:
        k = cpu_workers(host_info()["nproc"], N_GRID)
        v, dt, workers, host = cpu_sample(k, 0, N_GRID)
        cpu = {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle",
               "nproc": host["nproc"], "cpu_model": host["cpu_model"], "machine": host["machine"],
               "sample": f"{k} oracle right-hand-side evaluations of the {N_GRID}^3 TG field "
                         f"(FP64 numpy with the oracle's own FFT), one on each of {workers} "
                         f"single-threaded worker processes, {dt:.1f} s wall"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPES[args.precision],
           "data": "synthetic",
           "config": {"workload": workload_name(args), "grid": [n, n, n], "nu": nu,
                      "method": "BS5_ADAPTIVE" if args.mode == "step" else "rhs",
                      "rtol": TOL, "atol": TOL, "h0": H0, "precision": args.precision,
                      "forcing": forcing, "tiles": tiles,
                      "l2": "inputs larger than L2 (per right-hand side: "
                            f"{a['rhs_bytes'] / 1e9:.2f} GB algorithmic traffic)",
                      "parallelism": f"replicas{ws}"},
           "sim_time_per_gpu_s": sim_tot / (ms_max * 1e-3),
           "sim_time_advanced": sim, "rhs_evals": n_rhs, "t_end_state": i1.t,
           "accepted": i1.n_acc - i0.n_acc, "rejected": i1.n_rej - i0.n_rej,
           "rhs_hbm_frac_of_measured": a["rhs_hbm_frac_of_measured"],
           "rhs_hbm_frac_basis": "the five passes' algorithmic bytes per right-hand side over their "
                                 "CUDA-event time per right-hand side that does work",
           "rhs_rate_hbm_frac_of_measured": a["rhs_bytes"] * value / ws / 1e9 / peaks["hbm_gbs"],
           "step_hbm_frac_of_measured": a["step_hbm_frac_of_measured"],
           "e2e": e2e,
           "gpu_launches": launches,
           "kernels": a["kernels"],
           "roofline": a["roofline"],
           "forms": forms,
           "clocks": clk,
           "cpu_baseline": cpu}
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--forms", nargs="*", default=["fp32_mixed", "fp32", "fp32x2"],
                    choices=["fp64", "fp32_mixed", "fp32x2", "fp32"],
                    help="other arithmetic forms timed on the same field after the headline run "
                         "(step mode, one GPU); none with an empty list")
    ap.add_argument("--tiles", type=int, nargs=2, default=None,
                    help="y-pass variant and z-pass code instead of the autotuner's choice")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_mixed", "fp32x2", "fp32"])
    ap.add_argument("--flow", default="tg", choices=["tg", "hit"])
    ap.add_argument("--mode", default="step", choices=["step", "rhs"])
    ap.add_argument("--workload", default="single", choices=["single", "ensemble", "accuracy", "controllers"])
    ap.add_argument("--rt-shape", type=int, nargs=3, default=[128, 128, 256])
    ap.add_argument("--val-shape", type=int, nargs=3, default=[64, 64, 128],
                    help="grid of the controllers workload's validation problem (seed 13)")
    ap.add_argument("--val-width", type=float, default=0.1,
                    help="interface width of the validation problem")
    ap.add_argument("--ref-tol", type=float, default=1e-9)
    ap.add_argument("--ctrl-tols", type=float, nargs="+", default=[1e-5, 1e-6, 1e-7, 1e-8],
                    help="tolerance sweep of the controllers workload")
    ap.add_argument("--rk4-dt", type=float, default=0.02)
    ap.add_argument("--rk4-levels", type=int, default=4)
    ap.add_argument("--tols", type=float, nargs="+", default=[1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9])
    ap.add_argument("--dp5-tols", type=float, nargs="*", default=[1e-6, 1e-8])
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--t-end", type=float, default=0.5)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "accuracy":
        if args.t_end == 0.5:
            args.t_end = T_END
        return run_accuracy(args)
    if args.workload == "controllers":
        if args.t_end == 0.5:
            args.t_end = 5.0
        return run_controllers(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
