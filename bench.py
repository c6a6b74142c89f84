#!/usr/bin/env python
"""Benchmark of the pide2d time step on one GB300.

Workload (default): the large single solve -- put on the average, 4096^2
log grid (8192^2 padded transforms), NTS with alpha = 0.5, kappa = 0.5,
1024 time steps, fixed-point tol 1e-7, FP32-bulk transforms.  A "step" is
one theta time step of Algorithm 1 (SL preparation, one full B_w sweep and
the fixed-point loop, each iteration one B_w sweep plus the DST diffusion
solve).  Unit of work: one cell-iteration = one grid cell (N^2 per sweep)
through one application of B_w; a step with k fixed-point iterations
processes N^2 (k + 1) of them.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead
(on a bounded sample of the same workload).  Under torchrun (N > 1) every
rank runs an independent replica (the solve does not shard); value is the
sum of the units over the max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-iterations/s of 2D PIDE step vs FP64 plain at ≤1e-5 error; %HBM roofline"
UNIT = "cell-iterations/s"
FALLBACK_HBM_GBS = 6800.0


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=4096, help="grid size (default: the large 4096^2 workload)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the 512-pricing batch measurement")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    p.add_argument("--no-sweep", action="store_true", help="skip the FP32-bulk vs FP64 convergence sweep")
    p.add_argument("--no-fp64", action="store_true",
                   help="skip the FP64-mode solve of the same workload (the error of the FP32-bulk result)")
    p.add_argument("--no-paper", action="store_true",
                   help="skip the paper's own set-ups (price-space scheme, VG0 on the wide log domain)")
    p.add_argument("--host-loop", action="store_true",
                   help="drive the fixed-point loop from the host in the timed region too (one launch per "
                        "kernel, as the profilers see it)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(n):
    from paper_2511_02700_gb300.workloads import LARGE_FP32_4096, with_
    w = LARGE_FP32_4096
    if n != w.n:
        w = with_(w, name=f"large_fp32_{n}", n=n, steps=n // 4)
    return w


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        # raw samples go to $PIDE2D_CLOCKS_DIR (default: the temporary directory)
        out_dir = os.environ.get("PIDE2D_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"pide2d_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        sm = [c for c, _, _ in rows]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(m for _, m, _ in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- roofline
def algorithmic_bytes(cls, n, hcount=4):
    """Algorithmic HBM bytes of one launch of a kernel class, FP32-bulk mode
    (complex spectra 8 B, state 8 B double-float, R fields 4 B)."""
    P = 2 * n
    H = P // 2 + 1
    cells = n * n
    spec_full = (P + 2) * H * 8
    spec_n = n * H * 8
    wh = P * H * 8
    return {
        0: (8 * hcount + 8 + 16) * cells,                      # prep: V history, BV -> W, Y
        1: 16 * cells + spec_full,                             # row forward (difference): Y, V^{n-1} -> S
        2: 4 * cells + spec_n,                                 # row forward incr: D -> S
        3: spec_full + wh + spec_n,                            # column pass full
        4: spec_n + wh + spec_n,                               # column pass incr
        5: spec_n + 8 * cells + 8 * cells + 16 * cells + 4 * cells,   # inverse full: S, BV, BY, W+Y, E
        6: spec_n + 16 * cells + 4 * cells + 4 * cells,        # inverse incr: S, BY, D, E
        7: 8 * cells,                                          # column solve (E in, E out)
        8: 4 * cells + 16 * cells + 4 * cells + spec_n,        # row DST back (E, Y, D) + increment R2C rows
    }[cls]


KERNEL_NAMES = ["k_prep", "k_row_forward(full)", "k_row_forward(incr)", "k_col(full)", "k_col(incr)",
                "k_row_inverse(full)", "k_row_inverse(incr)", "k_col_solve", "k_dst_row+fwd"]
# the kernels of one fixed-point iteration (the B_w sweep of an increment fused with the DST solve)
ITERATION_KERNELS = (7, 8, 4, 6)
# algorithmic bytes of one cell-iteration of the FFT sweep alone (FP32, P = 2N, pruned R2C):
# read Y 4, two round trips of the N x (P/2+1) intermediate 32, read w^ 16, read W + write RHS 8
SWEEP_BYTES_PER_CELL = 60


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha256():
    """sha256 of the sources the ncu counters depend on: the time-loop kernels
    and the host code that sizes their launches."""
    csrc = os.path.join(ROOT, "paper_2511_02700_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("sweep_impl.cuh", "common.cuh", "state.cuh", "api.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def recorded_traffic(kernel, n):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources, else None.  Traffic grows with the cells
    processed, so a capture at another n is scaled by (n / n_captured)^2."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha256") != kernel_source_sha256():
        return None
    return float(e["dram_bytes_per_launch"]) * (n * n) / float(e["n"] ** 2)


# --------------------------------------------------------------------------- oracle arm
def host_cpu():
    """nproc and the CPU model of this host (lscpu, else /proc/cpuinfo)."""
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
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


def _oracle_replica(args):
    steps, warmup, n_sample = args
    return oracle_sample(steps, warmup, n_sample)


def oracle_sample_all_cores(steps, warmup, n_sample=512, procs=None):
    """The oracle sample on every host core: one single-threaded oracle
    process per core (spawned), all on the same sample; aggregate throughput
    = units of all processes over the slowest process's stepping time."""
    import multiprocessing as mp
    ncpu, _ = host_cpu()
    procs = procs or ncpu
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_replica, [(steps, warmup, n_sample)] * procs)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(r["units"] for r in res)
    t = max(r["seconds"] for r in res)
    return units / t, procs


def cpu_baseline_block(steps, warmup, n_sample=512, all_cores=True):
    """The oracle timed on this host: one core, and all cores as independent
    replicas; the line's value is the all-core figure."""
    ncpu, model = host_cpu()
    one = oracle_sample(steps, warmup, n_sample)
    out = dict(one)
    out.update({"value_1core": one["value"], "cores_available": ncpu, "cpu_model": model})
    if all_cores and ncpu > 1:
        v_all, procs = oracle_sample_all_cores(steps, warmup, n_sample)
        out.update({"value": v_all, "cores": procs, "value_all_cores": v_all,
                    "sample": one["sample"] + f"; all-core figure: {procs} concurrent single-threaded oracle "
                                              f"processes (spawned), one per core, on the same sample, units of all "
                                              f"processes over the slowest one's time"})
    out.pop("units", None)
    out.pop("seconds", None)
    return out


def oracle_sample(steps, warmup, n_sample=512):
    """FP64 CPU oracle on a bounded sample of the workload: same model,
    tolerance and scheme on an n_sample^2 grid; times `steps` time steps
    after `warmup` (the damped first step included in the warm-up)."""
    import oracle as O
    w = workload(4096)
    m = O.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    g = O.Grid(n_sample, half_width=w.half_width)
    c = O.Contract(O.PUT_AVG, w.strike, w.maturity)
    t0 = time.perf_counter()
    S = O.Scheme(m, g, c, n_sample // 4, theta=w.theta, tol=w.tol, sl_order=w.sl_order)
    it = S.iterate()
    setup = time.perf_counter() - t0
    for _ in range(max(1, warmup)):
        next(it)
    units = 0
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        try:
            _, k = next(it)
        except StopIteration:
            break
        units += n_sample * n_sample * (k + 1)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "units": units, "seconds": dt,
            "sample": f"FP64 oracle, {n_sample}^2 grid of the same model/tol, {done} time steps after "
                      f"{max(1, warmup)} warm-up steps ({dt:.1f} s; setup {setup:.1f} s); numpy/scipy "
                      "single-threaded FFT and sparse LU"}


def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cb = cpu_baseline_block(max(1, a.steps), max(1, a.warmup))
    w = workload(a.n)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "alpha": w.alpha, "tol": w.tol,
                       "oracle_sample_n": 512},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_over_ranks(ms, units, device=None):
    """Whole-job time and work over the ranks of the default process group:
    the slowest rank's milliseconds (MAX) and the units of all ranks (SUM).
    Without a process group (one GPU) the rank's own values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    uu = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


# --------------------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2511_02700_gb300 import binding as B
    from paper_2511_02700_gb300 import build as libbuild
    libbuild.build()
    w = workload(a.n)
    n = w.n
    prec = B.PIDE2D_FP32_BULK if w.precision == "fp32" else B.PIDE2D_FP64
    grid = B.make_grid(n, prec, w.sl_order, half_width=w.half_width)
    model = B.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    contract = B.make_contract(B.PIDE2D_PUT_AVG, w.strike, w.maturity)
    stream = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    s = B.Solver(grid, model, contract, w.steps, theta=w.theta, tol=w.tol, device=dev, stream=stream,
                 host_loop=a.host_loop)
    create_s = time.perf_counter() - t0
    if a.warmup + a.steps > w.steps:
        raise SystemExit("warmup + steps exceeds the workload's time steps")
    if a.warmup + 2 * a.steps > w.steps:
        raise SystemExit("warmup + 2 * steps exceeds the workload's time steps")
    for _ in range(a.warmup):
        s.step()
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    units = 0
    iters = []
    for _ in range(a.steps):
        k, r, st = s.step()
        iters.append(k)
        units += n * n * (k + 1)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    # kernels launched in the timed region.  Device loop: per step k_explicit + k_prep and the
    # difference sweep (5), setup and tally (2), per iteration col_solve, dst_row, check, col,
    # row_inverse (5).  Host loop: 5 per step, 4 per iteration.
    gpu_launches = sum(5 + 4 * k for k in iters) if a.host_loop else sum(7 + 5 * k for k in iters)
    # roofline pass: the next `steps` time steps with per-kernel CUDA events (host-driven loop,
    # one launch per kernel, so each launch can be bracketed)
    B.pide2d_profile(s.h, 1)
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    piters = []
    for _ in range(a.steps):
        k, r, st = s.step()
        piters.append(k)
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    prof_ms = pe0.elapsed_time(pe1)
    B.pide2d_profile(s.h, 0)
    kt = B.pide2d_profile_read(s.h)
    launches = [kt.launches[i] for i in range(9)]
    kms = [kt.ms[i] for i in range(9)]
    # aggregate over ranks
    t_max, units_all = aggregate_over_ranks(ms, units, dev)
    value = units_all / (t_max / 1e3)
    # roofline of the dominant kernel class
    top = max(range(9), key=lambda i: kms[i])
    bytes_per_launch = algorithmic_bytes(top, n)
    avg_ms = kms[top] / max(1, launches[top])
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    total_kms = sum(kms)
    roof = {"bound": "hbm", "kernel": KERNEL_NAMES[top], "achieved": achieved, "peak": peak,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(KERNEL_NAMES[top], n),
            "pass": f"{a.steps} time steps right after the timed region, host-driven loop with per-kernel "
                    f"CUDA events on the solver stream ({prof_ms / a.steps:.3f} ms/step there)",
            "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
            "share_of_kernel_time": kms[top] / total_kms if total_kms > 0 else None}
    # the whole fixed-point iteration: its four kernels' summed event time per iteration, against
    # their own algorithmic bytes and against the 60 B per cell of the FFT sweep alone
    n_it = launches[ITERATION_KERNELS[0]]
    if n_it:
        it_ms = sum(kms[i] for i in ITERATION_KERNELS) / n_it
        it_bytes = sum(algorithmic_bytes(i, n) for i in ITERATION_KERNELS)
        roof["iteration"] = {
            "kernels": [KERNEL_NAMES[i] for i in ITERATION_KERNELS], "ms_per_iteration": it_ms,
            "algorithmic_bytes": it_bytes, "achieved": it_bytes / (it_ms / 1e3) / 1e9,
            "frac": it_bytes / (it_ms / 1e3) / 1e9 / peak,
            "sweep_bytes_per_cell": SWEEP_BYTES_PER_CELL,
            "sweep_achieved": SWEEP_BYTES_PER_CELL * n * n / (it_ms / 1e3) / 1e9,
            "sweep_frac": SWEEP_BYTES_PER_CELL * n * n / (it_ms / 1e3) / 1e9 / peak,
            "note": "frac: the four kernels' own algorithmic bytes (DST solve and double-float state "
                    "included); sweep_frac: 60 B per cell-iteration for the FFT sweep alone, over the "
                    "same time, i.e. with the DST solve counted as overhead"}
    kernels = {KERNEL_NAMES[i]: {"launches": launches[i], "ms": round(kms[i], 3),
                                 "GBps": (algorithmic_bytes(i, n) * launches[i] / (kms[i] / 1e3) / 1e9)
                                 if kms[i] > 0 else None}
               for i in range(9) if launches[i]}
    # end to end: a fresh job from host inputs to host outputs through the C ABI
    e2e = None
    e2e_V = None
    if not a.no_e2e:
        e2e, e2e_V = run_e2e(B, torch, dev, grid, model, contract, w, a.warmup + a.steps)
    fp64 = None
    if not a.no_fp64 and e2e is not None and ws == 1:
        fp64 = run_fp64_plain(B, torch, dev, w, e2e["price"], e2e_V)
    s.close()
    if ws > 1:
        torch.distributed.barrier()
    if rank != 0:
        return
    cb = None
    if not a.no_cpu_baseline and ws == 1:
        cb = cpu_baseline_block(steps=6, warmup=1)
    batch = None if (a.no_batch or ws > 1) else run_batch(B, torch, dev)
    adjoint = None if (a.no_adjoint or ws > 1) else run_adjoint(B, torch, dev)
    sweep = None if (a.no_sweep or ws > 1) else run_sweep(B, torch, dev)
    paper = None if (a.no_paper or ws > 1) else run_paper_schemes(B, torch, dev)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "padded_fft": 2 * n, "alpha": w.alpha, "kappa": w.kappa,
                       "time_steps_total": w.steps, "tol": w.tol, "precision": "fp32-bulk (state double-float)",
                       "sl_order": w.sl_order, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "working set > L2 (inputs larger than the 129 MB L2, no flush)"},
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": gpu_launches,
            "error_vs_fp64": None if fp64 is None else {
                "price_rel": fp64["price_rel_err"], "roi_maxnorm_rel": fp64["roi_maxnorm_rel_err"],
                "bound": 1e-5, "against": "FP64-mode GPU solve of the same workload (fp64_plain)"},
            "fp64_plain": fp64,
            "clocks": ck, "fp_iters_per_step": iters, "create_s": create_s, "kernels": kernels,
            "batch": batch, "adjoint": adjoint, "convergence_sweep": sweep, "paper_schemes": paper,
            "loop": "host-driven fixed-point loop" if a.host_loop else
                    "device-side fixed-point loop (CUDA graph while-node), one host sync per time step"}
    print(json.dumps(line), flush=True)


def _job(B, w, payoff=0):
    prec = B.PIDE2D_FP64 if w.precision == "fp64" else B.PIDE2D_FP32_BULK
    grid = B.make_grid(w.n, prec, w.sl_order, half_width=w.half_width)
    model = B.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    contract = B.make_contract(payoff, w.strike, w.maturity)
    return grid, model, contract


def run_batch(B, torch, dev, lanes=256, fp64_sample=16):
    """The 512 seed-drawn pricings (N in {128, 256, 512}, FP32-bulk) through
    pide2d_batch_solve, wall time from the call to the prices on the host;
    then the first `fp64_sample` jobs again as plain FP64 GPU solves, for the
    price error and the FP64 throughput on the same GPU."""
    from paper_2511_02700_gb300.workloads import batch_draw, with_
    ws = batch_draw(512)
    jobs = []
    for w in ws:
        g, m, c = _job(B, w)
        jobs.append(B.make_job(g, m, c, w.steps, theta=w.theta, tol=w.tol))
    B.solve_batch(jobs[:lanes], lanes=lanes)              # warm-up: module load, streams
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    prices, sts, st = B.solve_batch(jobs, lanes=lanes)
    t1 = time.perf_counter()
    errs, cells64, t64 = [], 0.0, 0.0
    for w, p32 in zip(ws[:fp64_sample], prices[:fp64_sample]):
        w64 = with_(w, precision="fp64")
        g, m, c = _job(B, w64)
        torch.cuda.synchronize(dev)
        a0 = time.perf_counter()
        s = B.Solver(g, m, c, w64.steps, theta=w64.theta, tol=w64.tol, device=dev)
        p64, _, st64, _ = s.solve()
        a1 = time.perf_counter()
        s.close()
        errs.append(abs(p32 - p64) / max(abs(p64), 1e-300))
        cells64 += st64.cell_iters
        t64 += a1 - a0
    return {"workload": "batch_draw(512): N in {128,256,512}, N/4 steps, FP32-bulk, tol 1e-8",
            "loop": "one CUDA graph per chunk (while-node over theta steps around a while-node over "
                    "fixed-point iterations), one launch and one host wait per chunk",
            "tuning": st.tuning(), "create_s": st.create_s, "tune_s": st.tune_s, "loop_s": st.loop_s,
            "jobs": len(jobs), "lanes": lanes, "failures": st.failures, "wall_s": t1 - t0,
            "value": st.cell_iters / (t1 - t0), "unit": UNIT, "jobs_per_s": len(jobs) / (t1 - t0),
            "fp64_sample_jobs": fp64_sample, "price_max_rel_err_vs_fp64": max(errs),
            "fp64_plain_value": cells64 / t64, "fp64_plain_wall_s": t64,
            "note": "FP64 plain = the same jobs solved one by one in FP64 mode on the same GPU (create + solve)"}


def run_adjoint(B, torch, dev):
    """The adjoint workload at alpha 0.25 and 0.5 (run_adjoint_one each)."""
    from paper_2511_02700_gb300.workloads import ADJOINT_FP64_1024, with_
    return [run_adjoint_one(B, torch, dev, with_(ADJOINT_FP64_1024, alpha=a_)) for a_ in (0.25, 0.5)]


def run_adjoint_one(B, torch, dev, w):
    """Adjoint on the 1024^2, 256-step FP64 workload: forward solve with
    checkpoints every 16 steps, then pide2d_adjoint for the six workload
    parameters; checked against FP64 central differences (step 1e-4) of the
    CUDA path's prices.  The FP32-bulk adjoint is timed beside it."""
    from paper_2511_02700_gb300.workloads import ADJOINT_INTERVAL, with_
    names = B.SUBORDINATED_BM_PARAMS
    out = {"workload": f"{w.name}: alpha {w.alpha}, {w.steps} steps, tol {w.tol}, checkpoint interval "
                       f"{ADJOINT_INTERVAL}", "params": list(names)}

    def forward_adjoint(wx):
        g, m, c = _job(B, wx)
        wl = B.make_workload(wx.alpha, wx.kappa, wx.beta, wx.sigma, wx.corr, wx.r)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s = B.Solver(g, m, c, wx.steps, theta=wx.theta, tol=wx.tol, device=dev)
        s.record(interval=ADJOINT_INTERVAL, ndirs=6)
        price, _, st, _ = s.solve()
        t1 = time.perf_counter()
        grad, ast = s.adjoint_workload(wl)
        t2 = time.perf_counter()
        s.close()
        return price, grad, t1 - t0, t2 - t1, st.cell_iters

    def plain(wx):
        g, m, c = _job(B, wx)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s = B.Solver(g, m, c, wx.steps, theta=wx.theta, tol=wx.tol, device=dev)
        price, _, st, _ = s.solve()
        t1 = time.perf_counter()
        s.close()
        return price, t1 - t0, st.cell_iters

    p64, t_plain, cells = plain(w)
    price, grad, t_fwd, t_adj, _ = forward_adjoint(w)
    out.update({"price": price, "grad": dict(zip(names, grad)), "fp64_plain_solve_s": t_plain,
                "fp64_forward_with_checkpoints_s": t_fwd, "fp64_adjoint_s": t_adj,
                "adjoint_over_plain_solve": t_adj / t_plain,
                "fp64_plain_value": cells / t_plain, "unit": UNIT})
    # FP64 central differences of the CUDA path's prices
    eps = 1e-4
    base = {"sigma1": w.sigma[0], "sigma2": w.sigma[1], "corr": w.corr, "kappa": w.kappa,
            "beta1": w.beta[0], "beta2": w.beta[1]}
    fd = []
    for nm in names:
        pr = []
        for sgn in (1.0, -1.0):
            v = dict(base)
            v[nm] += sgn * eps
            wx = with_(w, sigma=(v["sigma1"], v["sigma2"]), corr=v["corr"], kappa=v["kappa"],
                       beta=(v["beta1"], v["beta2"]))
            pr.append(plain(wx)[0])
        fd.append((pr[0] - pr[1]) / (2 * eps))
    scale = max(abs(x) for x in fd)
    out["fd_grad"] = dict(zip(names, fd))
    out["fd_max_abs_err_over_max_grad"] = max(abs(a_ - b_) for a_, b_ in zip(grad, fd)) / scale
    # FP32-bulk forward + adjoint of the same workload
    w32 = with_(w, precision="fp32", tol=1e-8)
    p32, g32, t_fwd32, t_adj32, _ = forward_adjoint(w32)
    out.update({"fp32_bulk_price_rel_err_vs_fp64": abs(p32 - p64) / abs(p64),
                "fp32_bulk_forward_with_checkpoints_s": t_fwd32, "fp32_bulk_adjoint_s": t_adj32,
                "fp32_bulk_grad_max_abs_err_over_max_grad": max(abs(a_ - b_) for a_, b_ in zip(g32, grad)) / scale})
    return out


def _bilinear_at(x, V, p1, p2):
    """V[m2, m1] on the grid x (both axes) at (p1, p2), linear in each axis."""
    import numpy as np
    def w(p):
        i = int(np.searchsorted(x, p, side="right")) - 1
        i = min(max(i, 0), len(x) - 2)
        t = (p - x[i]) / (x[i + 1] - x[i])
        return i, t
    i1, t1 = w(p1)
    i2, t2 = w(p2)
    return float((1 - t2) * ((1 - t1) * V[i2, i1] + t1 * V[i2, i1 + 1])
                 + t2 * ((1 - t1) * V[i2 + 1, i1] + t1 * V[i2 + 1, i1 + 1]))


def run_paper_schemes(B, torch, dev):
    """The paper's own Sec. 4 set-ups through the CUDA path, each timed end to
    end (handle creation with the device precompute, all time steps, values
    back): Algorithm 1 in price space on the sinh grid (FP64 where the
    transform fits, N_t = N_x / 2, tol 1e-7; VG1 and NIG1), and VG0 on the wide log domain (half-width 11.5,
    FP32-bulk, 2048^2, N/2 steps, tol 1e-8).  Each reports the price at (K, K)
    beside the paper's Table 4 value (N_x = 800)."""
    from paper_2511_02700_gb300.workloads import PAPER_SETS
    res = {"price_space": []}
    for name in ("VG1", "NIG1"):
        ps = PAPER_SETS[name]
        model = B.make_model(ps.alpha, ps.delta, ps.lam, ps.eta, ps.rho, ps.r)
        for nx in (160, 320):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            x, n_z, h_z, nym, nyp = B.price_sinh_grid(nx, ps.strike, ps.x_max_over_k * ps.strike, ps.z_max_iii)
            # FP64 transforms go up to length 4096; longer ones (NIG1 at N_x = 320) run in FP32-bulk
            prec = "fp64"
            try:
                pj = B.PriceJump(x, n_z, h_z, nym, nyp, model, precision=B.PIDE2D_FP64, device=dev)
            except B.PideError:
                prec = "fp32-bulk"
                pj = B.PriceJump(x, n_z, h_z, nym, nyp, model, precision=B.PIDE2D_FP32_BULK, device=dev)
            V, st, status = pj.solve(B.make_contract(B.PIDE2D_PUT_AVG, ps.strike, ps.maturity), nx // 2, tol=1e-7)
            V = V.cpu().numpy()
            wall = time.perf_counter() - t0
            pj.close()
            price = _bilinear_at(x, V, ps.strike, ps.strike)
            res["price_space"].append({
                "set": name, "n_x": nx, "precision": prec, "time_steps": nx // 2, "status": status, "wall_s": wall,
                "fp_iters_total": st.fp_iters_total, "cell_iterations_per_s": st.cell_iters / wall,
                "price_at_KK": price, "table4_at_KK": ps.table4_at_k, "diff": price - ps.table4_at_k})
    ps = PAPER_SETS["VG0"]
    n, hw = 2048, 11.5
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    grid = B.make_grid(n, B.PIDE2D_FP32_BULK, 3, half_width=hw)
    model = B.make_model(ps.alpha, ps.delta, ps.lam, ps.eta, ps.rho, ps.r)
    s = B.Solver(grid, model, B.make_contract(B.PIDE2D_PUT_AVG, ps.strike, ps.maturity), n // 2, tol=1e-8,
                 device=dev)
    price, _, st, _ = s.solve()
    wall = time.perf_counter() - t0
    s.close()
    res["vg0_wide_log_domain"] = {
        "n": n, "half_width": hw, "time_steps": n // 2, "precision": "fp32-bulk", "wall_s": wall,
        "fp_iters_total": st.fp_iters_total, "cell_iterations_per_s": st.cell_iters / wall,
        "price_at_KK": price, "table4_at_KK": ps.table4_at_k, "diff": price - ps.table4_at_k}
    return res


def run_sweep(B, torch, dev):
    """The convergence sweep: alpha in {0.25, 0.5, 0.75} x N in {256, 512,
    1024}, N/4 steps, tol 1e-8, solved in FP64 and in FP32-bulk on the GPU.
    Per case: the price at S0, the FP32-bulk error against FP64 at S0 and in
    max-norm over the region of interest (S_i <= 3K), and the wall times;
    per alpha the observed order of the FP64 price from the three grids."""
    import math
    from paper_2511_02700_gb300.workloads import convergence_sweep
    cases = []
    by_alpha = {}
    for w64, w32 in zip(convergence_sweep("fp64"), convergence_sweep("fp32")):
        out = {}
        for tag, w in (("fp64", w64), ("fp32", w32)):
            g, m, c = _job(B, w)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            s = B.Solver(g, m, c, w.steps, theta=w.theta, tol=w.tol, device=dev)
            price, V, st, _ = s.solve(values=True)
            torch.cuda.synchronize(dev)
            out[tag] = (price, V.cpu().numpy(), time.perf_counter() - t0, st.cell_iters)
            s.close()
        n = w64.n
        h = 2 * w64.half_width / n
        sg = math.log(w64.strike) - w64.half_width + h * np.arange(n + 1)
        roi1 = np.exp(sg) <= 3 * w64.strike
        roi = np.outer(roi1, roi1)
        roi[0, :] = roi[-1, :] = roi[:, 0] = roi[:, -1] = False
        p64, V64, t64, c64 = out["fp64"]
        p32, V32, t32, c32 = out["fp32"]
        cases.append({"alpha": w64.alpha, "n": n, "steps": w64.steps, "price_fp64": p64, "price_fp32": p32,
                      "price_rel_err": abs(p32 - p64) / abs(p64),
                      "roi_maxnorm_rel_err": float(np.abs(V32 - V64)[roi].max() / np.abs(V64[roi]).max()),
                      "fp64_s": t64, "fp32_s": t32, "fp64_value": c64 / t64, "fp32_value": c32 / t32})
        by_alpha.setdefault(w64.alpha, []).append(p64)
    orders = {}
    for a_, ps in by_alpha.items():
        d1, d2 = ps[1] - ps[0], ps[2] - ps[1]
        orders[str(a_)] = math.log2(abs(d1 / d2)) if d2 != 0 else None
    return {"cases": cases, "fp64_observed_order_256_512_1024": orders,
            "max_price_rel_err": max(c["price_rel_err"] for c in cases),
            "max_roi_maxnorm_rel_err": max(c["roi_maxnorm_rel_err"] for c in cases)}


def run_e2e(B, torch, dev, grid, model, contract, w, steps):
    """One complete pricing through the C ABI, as a user calls it:
    pide2d_create from host structs (device precompute), pide2d_solve over all
    the workload's time steps, V^{N_t} copied to a pinned host buffer and the
    price returned to the host; cell-iterations over wall time.  The
    fixed-point loop runs on the device, so the host waits once, at the end."""
    n = grid.n
    nbytes = B.pide2d_workspace_bytes(grid)
    wsb = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = (wsb.data_ptr() + 255) & ~255
    host = torch.empty(((n + 1) * (n + 1),), dtype=torch.float64, pin_memory=True)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    opts = B.pide2d_options()
    opts.kmax, opts.damping = 100, 1
    h = B.pide2d_create(grid, model, contract, w.theta, w.maturity / w.steps, w.tol, opts, base, nbytes,
                        stream.cuda_stream)
    price, stats, st = B.pide2d_solve(h, host.data_ptr())
    t1 = time.perf_counter()
    B.pide2d_destroy(h)
    nsteps = stats.steps_done
    # create: quadrature nodes and parameter blocks in, rates and the sin^2 table out and back;
    # solve: the loop statistics (48 B), V and the price out
    h2d = 2 * (10 + 6 + 32 + 16 + 4) * 8 + (n + 1) * 4
    d2h = (n + 1) * (n + 1) * 8 + 9 * 8 + (n + 1) * 8 + 48 + 8
    return ({"value": stats.cell_iters / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d / nsteps,
             "d2h_bytes_per_step": d2h / nsteps, "steps": nsteps, "wall_s": t1 - t0, "price": price,
             "fp_iters_total": stats.fp_iters_total,
             "includes": "pide2d_create (device precompute) + pide2d_solve over all time steps + V to pinned host"},
            host.numpy().reshape(n + 1, n + 1))


def roi_mask(n, half_width, strike):
    """Nodes with S_i <= 3K in both axes (the region of interest), boundary excluded."""
    h = 2 * half_width / n
    sg = math.log(strike) - half_width + h * np.arange(n + 1)
    m1 = np.exp(sg) <= 3 * strike
    roi = np.outer(m1, m1)
    roi[0, :] = roi[-1, :] = roi[:, 0] = roi[:, -1] = False
    return roi


def run_fp64_plain(B, torch, dev, w, price32, V32):
    """The same workload solved in FP64 mode on the same GPU (create + all
    steps + V back), timed end to end; the FP32-bulk result's error against it
    at S0 and in max-norm over the region of interest."""
    grid = B.make_grid(w.n, B.PIDE2D_FP64, w.sl_order, half_width=w.half_width)
    model = B.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    contract = B.make_contract(B.PIDE2D_PUT_AVG, w.strike, w.maturity)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s = B.Solver(grid, model, contract, w.steps, theta=w.theta, tol=w.tol, device=dev)
    p64, V64, st, status = s.solve(values=True)
    V64 = V64.cpu().numpy()
    t1 = time.perf_counter()
    s.close()
    roi = roi_mask(w.n, w.half_width, w.strike)
    return {"price": p64, "status": status, "wall_s": t1 - t0, "value": st.cell_iters / (t1 - t0), "unit": UNIT,
            "fp_iters_total": st.fp_iters_total,
            "price_rel_err": abs(price32 - p64) / abs(p64),
            "roi_maxnorm_rel_err": float(np.abs(V32 - V64)[roi].max() / np.abs(V64[roi]).max()),
            "includes": "pide2d_create + pide2d_solve (FP64 mode, device loop) + V to the host"}


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
