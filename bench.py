#!/usr/bin/env python
"""ETDM energy+gradient evaluations per second on one GB300 (or N replicas).

Workload: the 96-atom water-like box (32 triatomic units, M = 256 s-Gaussians,
N = 128 doubly occupied orbitals, 96^3 grid over a 9.9 A cell, r_c = 4 A,
A_ov ~ N(0, 0.02)), synthetic inputs standing in for the paper's liquid-water
snapshots.  One step is one ETDM iteration through the C ABI
(etdm_minimize with one step: the energy+gradient at the current point, the
L-BFGS direction with the Eq. 33 preconditioner, and the line search, whose
trials are further evaluations); `value` counts every energy+gradient
evaluation made in the timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the path has no
exchange step); value = all evaluations / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ETDM energy+gradient evals/sec vs plain FP64 GPU path at |dE|<1e-6 Ha"
WORKLOADS = {
    "water32": "water32: 96 atoms, M=256, N=128, 96^3 grid, 9.9 A box, r_c=4 A",
    "small": "small molecule: 8 atoms, M=16, N=4, 32^3 grid, 6.4 A box",
    "water576": "water576: 1728 atoms, M=4608, N=2304, 192^3 grid, 25 A box, r_c=3.5 A",
}
WORKLOAD = WORKLOADS["water32"]


def workload_system(name):
    import etdm_synth as synth
    return {"water32": synth.config_water32, "small": synth.config_small_molecule,
            "water576": synth.config_water576}[name]()


FP64_PEAK_TFLOPS = 1.25      # nominal FP64 rate of a GB300 (no measured figure)
HBM_FALLBACK_GBS = 6800.0
BF16_FALLBACK_TFLOPS = 1900.0


def oracle_threads():
    """Threads the oracle's BLAS calls run on: threadpoolctl's count where it is
    installed, else OpenBLAS's environment variables in its own order of
    precedence, else the CPUs this process may run on (torchrun sets
    OMP_NUM_THREADS=1 for its workers)."""
    ncpu = len(os.sched_getaffinity(0))
    try:
        from threadpoolctl import threadpool_info
        n = [i["num_threads"] for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except ImportError:
        pass
    for k in ("OPENBLAS_NUM_THREADS", "GOTO_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(k, "")
        if v.isdigit() and int(v) > 0:
            return min(int(v), ncpu)
    return ncpu


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS, "bf16_tflops": BF16_FALLBACK_TFLOPS}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:  # no nvidia-smi: no clock record, and no file left behind
            os.unlink(self.path)
            self.proc, self.path = None, None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_baseline(d, budget_s=20.0, max_evals=6, workload=None):
    """The oracle as it stands on this host's cores: energy+gradient evaluations
    of the same workload (set-up not timed)."""
    workload = workload or WORKLOAD
    from oracle.etdm_oracle import Oracle
    o = Oracle(d)
    o.reference()
    t0 = time.perf_counter()
    n = 0
    a = d["a0"]
    while n < max_evals:
        o.energy_grad(a)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "evals/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": f"{n} oracle energy+gradient evaluations of {workload} at A_ov = a0 "
                      "(numpy FP64; basis matrix and reference set up before timing)"}


def run_reference(args):
    # the oracle arm uses neither a GPU nor a collective: under torchrun rank 0
    # alone runs it and the other ranks exit without work
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from oracle.etdm_oracle import Oracle
    d = workload_system(args.workload)
    o = Oracle(d)
    o.reference()
    a = d["a0"]
    for _ in range(args.warmup):
        o.energy_grad(a)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.energy_grad(a)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": oracle_threads(),
                         "kind": "oracle",
                         "sample": "each step: 1 oracle energy+gradient evaluation of "
                                   f"{WORKLOADS[args.workload]}"},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def captured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel source changed since that capture."""
    import hashlib
    src = os.path.join(ROOT, "paper_2101_12597_gb300", "csrc", "mixed.cu")
    summ = os.path.join(ROOT, "profiles", "traffic_water32.md")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for ln in open(summ):
            f = ln.split()
            if len(f) == 4 and f[0] == "traffic" and f[1] == kernel and f[3] == f"mixed.cu:{h}":
                return int(f[2])
    except OSError:
        pass
    return None


def run_ours(args):
    import torch

    import etdm_synth as synth
    from paper_2101_12597_gb300 import build as b
    from paper_2101_12597_gb300.etdm import ETDM

    world, rank, local = dist_setup(args.gpus)
    b.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    d = workload_system(args.workload)
    solver = ETDM(d, precision=args.precision, device=local)
    dims = solver.dims
    a = torch.tensor(d["a0"], dtype=torch.float64, device=dev)
    if args.profile_once:  # one evaluation after set-up, for profiler captures
        solver.energy_grad(a)
        torch.cuda.synchronize()
        solver.check()
        print(json.dumps({"profile_once": True, "precision": args.precision}))
        return
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    for _ in range(args.warmup):
        solver.minimize(a, 1)
    torch.cuda.synchronize()
    solver.set_profiling(True)
    solver.stage_times()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    total_ms, evals = 0.0, 0
    Es = []
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        barrier(world)
        torch.cuda.synchronize()
        ev0.record()
        E, al, tr = solver.minimize(a, 1)
        ev1.record()
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        evals += 1 + int(tr[1])
        Es.append(float(E[1]))
    clk = clocks.stop()
    stage_ms, stage_n, launches = solver.stage_times()
    solver.set_profiling(False)
    t_max = reduce_max(total_ms, world, dev)
    all_evals = reduce_sum(evals, world, dev)
    value = all_evals / (t_max / 1e3)

    # end to end through the host-buffer entry point (copies inside the region)
    a_host = np.ascontiguousarray(d["a0"])
    solver.energy_grad_host(a_host)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.energy_grad_host(a_host)
    e2e_dt = reduce_max(time.perf_counter() - t0, world, dev)
    nvar = dims["N"] * dims["V"]
    e2e = {"value": world * args.steps / e2e_dt, "unit": "evals/s",
           "h2d_bytes_per_step": 8 * nvar, "d2h_bytes_per_step": 8 * (nvar + 1)}

    # the plain FP64 GPU path on the same workload (the metric's denominator) and
    # the energy difference of the timed configuration against it
    E_run, _ = solver.energy_grad_host(a_host)
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        ref = ETDM(d, precision="fp64", device=local)
        E64, _ = ref.energy_grad_host(a_host)
        a64 = torch.tensor(d["a0"], dtype=torch.float64, device=dev)
        ref.minimize(a64, 1)
        n64, ms64 = 0, 0.0
        for _ in range(min(3, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            _, _, tr64 = ref.minimize(a64, 1)
            ev1.record()
            torch.cuda.synchronize()
            ms64 += ev0.elapsed_time(ev1)
            n64 += 1 + int(tr64[1])
        fp64 = {"value": n64 / (ms64 / 1e3), "unit": "evals/s", "evals_timed": n64,
                "dE_Ha": abs(E_run - E64)}
        ref.close()

    # roofline of the dominant grid pass
    peaks, src = measured_peaks()
    dom = max(("rho", "vmat"), key=lambda k: stage_ms[k])
    per_launch_ms = stage_ms[dom] / max(1, stage_n[dom])
    flops = 2.0 * dims["sum_npt2"]  # one multiply-add per (point, mu, nu) within r_c
    achieved = flops / (per_launch_ms * 1e-3) / 1e12
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": f"{dom}_fp64 (FP64 DFMA)",
                "peak_source": "nominal FP64 rate of a GB300 (no measured FP64 figure)"}
    else:
        # the stage is timed inside a long step: the sustained BF16 figure
        pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", BF16_FALLBACK_TFLOPS))
        nu = solver.get_array("tile_nu_tc").astype(np.int64)  # functions per 128-point tile
        if dom == "vmat":  # 8 slice products per 16-point K step of a V group (runs of
            # consecutive tiles), M = 128 rows, N = the group's union list padded to 16
            t0 = solver.get_array("vgroup_t0").astype(np.int64)
            gnu = solver.get_array("vgroup_nu").astype(np.int64)
            npad = np.maximum(16, ((gnu + 15) // 16) * 16)
            executed = float((8 * 2.0 * 128 * npad * 128 * np.diff(t0)).sum())
        else:  # 9 slice products per 16-function K step, N = occupied orbitals padded to 32
            nocc = dims["N"]
            nmpad = sum(min(128, nocc - m0) for m0 in range(0, nocc, 128))
            nmpad = max(32, ((nmpad + 31) // 32) * 32)
            ksteps = np.maximum(1, (nu + 15) // 16)
            executed = float((9 * 2.0 * 128 * nmpad * 16 * ksteps).sum())
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk, "traffic": captured_traffic(f"{dom}_tc_kernel"),
                "kernel": f"{dom}_tc_kernel",
                "peak_source": f"{src} dense bf16" + (" (sustained)" if "bf16_tflops_sustained" in peaks else ""),
                "executed_tflops": executed / (per_launch_ms * 1e-3) / 1e12,
                "executed_frac": executed / (per_launch_ms * 1e-3) / 1e12 / pk}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": args.precision,
                   "parallelism": f"replicas{world}",
                   "l2": "flushed (512 MB write) before every timed step",
                   "evals_timed": int(all_evals), "E_last": Es[-1] if Es else None,
                   "stage_ms_per_launch": {k: stage_ms[k] / max(1, stage_n[k]) for k in stage_ms},
                   "M": dims["M"], "N": dims["N"], "grid_points": dims["G"],
                   "sum_npt2": dims["sum_npt2"], "fp64_path": fp64,
                   "E_run_Ha": E_run},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline and args.workload != "water576":
        line["cpu_baseline"] = cpu_baseline(d, workload=WORKLOADS[args.workload])
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="water32",
                    help="water32 (the metric's configuration), the 8-atom molecule, or "
                         "water576 (no CPU oracle baseline: its evaluation takes hours)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--profile-once", action="store_true",
                    help="set up, run one energy+gradient evaluation, exit (for ncu)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
