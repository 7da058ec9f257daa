#!/usr/bin/env python
"""ETDM energy+gradient evaluations per second on one GB300 (or N replicas).

Default workload: the liquid-water-sized box (576 triatomic units, 1728 atoms,
M = 4608 s-Gaussians, N = 2304 doubly occupied orbitals, 192^3 grid over a
25 A cell, r_c = 3.5 A), K L-BFGS steps of one ETDM minimization from the
seed-2 perturbed start A_ov ~ N(0, 0.01): synthetic inputs standing in for the
paper's liquid-water snapshots.  The K timed steps are one etdm_minimize call
through the C ABI (per step the L-BFGS direction with the Eq. 33
preconditioner and the line search, whose trials are energy+gradient
evaluations); `value` counts every energy+gradient evaluation in it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload water576|water32|small|molecules148|crystal64]

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
    "water576": "water576: 1728 atoms, M=4608, N=2304, 192^3 grid, 25 A box, r_c=3.5 A",
    "water32": "water32: 96 atoms, M=256, N=128, 96^3 grid, 9.9 A box, r_c=4 A",
    "water216": "water216: 648 atoms, M=1728, N=864, 128^3 grid, 18.03 A box, r_c=3.5 A",
    "small": "small molecule: 8 atoms, M=16, N=4, 32^3 grid, 6.4 A box",
    "molecules148": "molecules148: 148 molecules of 2-20 atoms (M 4-60), each on its own "
                    "48^3 grid over a 9.6 A box, r_c=4 A, evaluated as one batch",
    "crystal64": "crystal64: 64 atoms, M=512, 8 k-points (2x2x2 Monkhorst-Pack), 256 "
                 "electrons, kT=0.1 eV, 56^3 grid over an 11.2 A cell, r_c=4 A, full "
                 "complex A(k) per k-point",
}
# workloads whose per-evaluation operands exceed the 129 MB L2, so the timed
# steps run back to back: on the mixed path the resident basis slices (water32:
# 1.3 GB streamed per evaluation); on the FP64 path, which recomputes the basis
# from small tables, its dense M x M matrices (water216: 24 MB each, water576:
# 170 MB).  The other runs flush L2 before every timed step.
LARGE = {"water576", "water216", "water32"}
LARGE_FP64 = {"water576", "water216"}


def runs_back_to_back(workload, precision):
    """True where the inputs of a timed step exceed L2 (no flush between steps)."""
    return workload in (LARGE_FP64 if precision == "fp64" else LARGE)


def workload_system(name):
    import etdm_synth as synth
    return {"water32": synth.config_water32, "small": synth.config_small_molecule,
            "water576": synth.config_water576, "water216": synth.config_water216,
            "molecules148": synth.config_molecules148,
            "crystal64": synth.config_crystal64}[name]()


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


def _plane_sample_setup(d):
    """An oracle instance of the workload (basis streamed plane by plane, no
    reference orbitals: they need a full pass over the grid) with a fixed
    symmetric D and potential of the workload's sizes; the timing of the
    oracle's grid arithmetic does not depend on their values."""
    from oracle.etdm_oracle import Oracle
    o = Oracle(d, cache_x=False)
    rng = np.random.default_rng(0)
    C = rng.normal(size=(o.M, o.N)) / math.sqrt(o.M)
    D = 2.0 * C @ C.T
    v = rng.normal(size=o.G)
    return o, D, v


def _plane_sample(o, D, v, i):
    """Seconds the oracle takes for one x-plane of an evaluation's grid work:
    the basis on the plane (Eq. 3), the density there (Eq. 2) and the plane's
    part of the potential matrix (Eq. 11)."""
    per = int(o.n[1] * o.n[2])
    t0 = time.perf_counter()
    Xp = o.basis_plane(i)
    o.density_plane(Xp, D)
    o.potential_plane(Xp, v[i * per:(i + 1) * per])
    return time.perf_counter() - t0


PLANE_SAMPLE = ("the oracle's grid work (basis values, density, potential-matrix part) "
                "on {k} of the {n} x-planes of {w}, scaled by {n}/{k} to one evaluation; "
                "the dense steps (exp of A by eigendecomposition, products of M x M "
                "matrices) and the FFTs are left out: they are under 1% of an oracle "
                "evaluation at this size")


def cpu_baseline(d, workload, name, budget_s=20.0, max_evals=6):
    """The oracle as it stands on this host's cores.  Whole energy+gradient
    evaluations of the workload (set-up not timed), or, for the 192^3 water
    box (hours per oracle evaluation), a sample of x-planes of its grid work."""
    if name == "water576":
        o, D, v = _plane_sample_setup(d)
        t, k = 0.0, 0
        while k < int(o.n[0]) and (k == 0 or t < budget_s / 2):
            t += _plane_sample(o, D, v, k)
            k += 1
        n = int(o.n[0])
        return {"value": 1.0 / (t / k * n), "unit": "evals/s", "cores": oracle_threads(),
                "kind": "oracle", "sample": PLANE_SAMPLE.format(k=k, n=n, w=workload)}
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
    d = workload_system(args.workload)
    w = WORKLOADS[args.workload]
    if args.workload == "water576":
        # each step: one x-plane of the oracle's grid work, scaled to a whole
        # evaluation (an oracle evaluation of this box takes hours)
        o, D, v = _plane_sample_setup(d)
        n = int(o.n[0])
        for k in range(args.warmup):
            _plane_sample(o, D, v, k % n)
        t = sum(_plane_sample(o, D, v, (args.warmup + k) % n) for k in range(args.steps))
        dt = t * n  # seconds of the K whole evaluations the samples stand for
        sample = PLANE_SAMPLE.format(k=1, n=n, w=w) + " (one x-plane per step)"
    elif args.workload == "crystal64":
        # each step: one x-plane of one k-point's oracle grid work, scaled to a
        # whole evaluation (8 k-points; an oracle evaluation takes minutes)
        from oracle.etdm_kpoints import BlochOracle
        o = BlochOracle(d, cache_x=False)
        rng = np.random.default_rng(0)
        C = rng.normal(size=(o.M, o.M)) + 1j * rng.normal(size=(o.M, o.M))
        D = (C @ C.conj().T) / o.M
        vv = rng.normal(size=o.G)
        n = int(o.n[0])
        for k in range(args.warmup):
            _kplane_sample(o, D, vv, k % n)
        t = sum(_kplane_sample(o, D, vv, (args.warmup + k) % n) for k in range(args.steps))
        dt = t * n * o.nk
        sample = KPLANE_SAMPLE.format(k=1, n=n, nk=o.nk, w=w) + " (one x-plane per step)"
    elif args.workload == "molecules148":
        # each step: one molecule's oracle evaluation, the molecules in turn
        # (set-up not timed); the unit is molecule evaluations per second
        from oracle.etdm_oracle import Oracle
        n = args.warmup + args.steps
        os_ = [Oracle(d[k % len(d)]) for k in range(n)]
        for o in os_:
            o.reference()
        for k in range(args.warmup):
            os_[k].energy_grad(d[k % len(d)]["a0"])
        t0 = time.perf_counter()
        for k in range(args.warmup, n):
            os_[k].energy_grad(d[k % len(d)]["a0"])
        dt = time.perf_counter() - t0
        sample = (f"each step: 1 oracle energy+gradient evaluation of one molecule of {w}, "
                  "molecules in turn")
    else:
        from oracle.etdm_oracle import Oracle
        o = Oracle(d)
        o.reference()
        a = d["a0"]
        for _ in range(args.warmup):
            o.energy_grad(a)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            o.energy_grad(a)
        dt = time.perf_counter() - t0
        sample = f"each step: 1 oracle energy+gradient evaluation of {w}"
    v = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w, "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": oracle_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def captured_traffic(kernel, workload, doublings=None):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summaries (lines `traffic <kernel> <bytes> <source>:<sha256[:16]> <workload>`,
    optionally followed by `doublings=<j>` for the dense chains, whose product
    count depends on it), or None when the kernel's source changed since that
    capture or the capture ran another number of doublings."""
    import glob
    import hashlib
    for summ in sorted(glob.glob(os.path.join(ROOT, "profiles", "traffic_*.md"))):
        try:
            for ln in open(summ):
                f = ln.split()
                if len(f) not in (5, 6) or f[0] != "traffic" or f[1] != kernel or f[4] != workload:
                    continue
                if len(f) == 6 and f[5] != f"doublings={doublings}":
                    continue
                src, h = f[3].split(":")
                path = os.path.join(ROOT, "paper_2101_12597_gb300", "csrc", src)
                if hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] == h:
                    return int(f[2])
        except (OSError, ValueError):
            pass
    return None


def dense_macs(M, N, V, J):
    """Multiply-adds of the dense chains of one evaluation (Eq. 7, 37 and the
    reverse pass), product by product as the kernels run them: forward P, Q^2,
    Q^3, Q^4, the two Paterson-Stockmeyer steps of cos and sin (one product
    each), k and s, J doublings of two products, U_vo, O = C0 U, then T O
    (mixed) or D = 2 O O^T; reverse 4 H O (4 V O), C0^T Gbar, the two products
    at U_vo, J reverse doublings of three products (symmetric cotangents),
    12 N^3 of the series' reverse and the one product of g."""
    n3 = float(N) ** 3
    fwd = 2.0 * N * N * V + (7 + 2 * J) * n3 + 2.0 * M * M * N
    rev = 2.0 * M * M * N + 3.0 * N * N * V + (12 + 3 * J) * n3
    return fwd, rev


def run_ours(args):
    import torch

    from paper_2101_12597_gb300 import build as b
    from paper_2101_12597_gb300.etdm import ETDM

    world, rank, local = dist_setup(args.gpus)
    b.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    d = workload_system(args.workload)
    solver = ETDM(d, precision=args.precision, device=local, dense_tc=args.dense_tc)
    dims = solver.dims
    a0 = torch.tensor(d["a0"], dtype=torch.float64, device=dev)
    if args.profile_once:  # one evaluation after set-up, for profiler captures
        solver.energy_grad(a0)
        torch.cuda.synchronize()
        solver.check()
        print(json.dumps({"profile_once": True, "precision": args.precision}))
        return
    large = runs_back_to_back(args.workload, args.precision)
    flush = None if large else torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    # warm-up: W steps of a minimization from the start point, then the memory
    # is erased and the timed run starts again from the same point
    a = a0.clone()
    if args.warmup:
        solver.minimize(a, args.warmup)
    torch.cuda.synchronize()
    solver.lbfgs_reset()
    a = a0.clone()
    solver.set_profiling(True)
    solver.stage_times()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed region
    if large:  # K steps of one minimization, back to back
        barrier(world)
        torch.cuda.synchronize()
        ev0.record()
        E_h, al_h, tr_h = solver.minimize(a, args.steps)
        ev1.record()
        torch.cuda.synchronize()
        total_ms = ev0.elapsed_time(ev1)
        evals = int(tr_h.sum())
        E_last = float(E_h[-1])
    else:  # one step per call, the L2 flushed before each
        total_ms, evals = 0.0, 0
        E_h = None
        for k in range(args.steps):
            flush.zero_()
            barrier(world)
            torch.cuda.synchronize()
            ev0.record()
            E1, al1, tr1 = solver.minimize(a, 1)
            ev1.record()
            torch.cuda.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            evals += int(tr1[1]) + (1 if k == 0 else 0)
            E_last = float(E1[1])
        # each call re-evaluates its start point (the point the previous call
        # accepted); only the first of those counts as new work
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    stage_ms, stage_n, launches = solver.stage_times()
    solver.set_profiling(False)
    J = int(solver.get_array("doublings")[0])
    t_max = reduce_max(total_ms, world, dev)
    all_evals = reduce_sum(evals, world, dev)
    value = all_evals / (t_max / 1e3)

    # end to end through the host-buffer entry point (copies inside the region)
    a_host = np.ascontiguousarray(d["a0"])
    solver.energy_grad_host(a_host)
    torch.cuda.synchronize()
    n_e2e = min(args.steps, 10) if large else args.steps
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        E_run, _ = solver.energy_grad_host(a_host)
    e2e_dt = reduce_max(time.perf_counter() - t0, world, dev)
    nvar = dims["N"] * dims["V"]
    e2e = {"value": world * n_e2e / e2e_dt, "unit": "evals/s",
           "h2d_bytes_per_step": 8 * nvar, "d2h_bytes_per_step": 8 * (nvar + 1),
           "evals": n_e2e}

    # the plain FP64 GPU path on the same workload (the metric's denominator) and
    # the energy difference of the timed configuration against it
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        ref = ETDM(d, precision="fp64", device=local)
        E64, _ = ref.energy_grad_host(a_host)
        a64 = a0.clone()
        torch.cuda.synchronize()
        k64 = min(3, args.steps)
        ev0.record()
        _, _, tr64 = ref.minimize(a64, k64)
        ev1.record()
        torch.cuda.synchronize()
        n64 = int(tr64.sum())
        fp64 = {"value": n64 / (ev0.elapsed_time(ev1) / 1e3), "unit": "evals/s",
                "evals_timed": n64, "steps_timed": k64, "dE_Ha": abs(E_run - E64)}
        ref.close()

    # roofline of the dominant kernel (the stage with the most time per evaluation)
    peaks, src = measured_peaks()
    per_eval = {k: stage_ms[k] / max(1, stage_n[k]) for k in stage_ms}
    mixed = args.precision == "mixed"
    M, N, V = dims["M"], dims["N"], dims["V"]
    fwd, rev = dense_macs(M, N, V, J)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    # float-pair multiply-add: 12 FP32 instructions, each one lane-cycle
    pair_peak = 152 * 128 * sm_mhz * 1e6 * 2.0 / 12.0 / 1e12
    pk_s = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", BF16_FALLBACK_TFLOPS))
    pk_src = f"{src} dense bf16" + (" (sustained)" if "bf16_tflops_sustained" in peaks else "")

    def dense_roof(dom):
        if not per_eval.get(dom, 0.0) > 0.0:
            return None
        flops = 2.0 * (fwd if dom == "dense_fwd" else rev)
        achieved = flops / (per_eval[dom] * 1e-3) / 1e12
        kern = "dense_forward_kernel" if dom == "dense_fwd" else "dense_reverse_kernel"
        # the float-pair products go to the tensor cores from 2^26 multiply-adds
        # on (every product of the chains at this size when the smallest does)
        on_tc = mixed and (args.dense_tc == 1 or
                           (args.dense_tc == 0 and N * N * min(N, V) >= 1 << 26))
        if on_tc:
            kern = kern.replace("_kernel", "_tc_kernel")
            # executed: 15 BF16 slice products per multiply-add, the outputs
            # padded to 128 x 64 tiles and K to 16
            pad = (lambda x, q: -(-x // q) * q)
            ex_fwd, ex_rev = dense_macs(pad(M, 128), pad(N, 64), pad(V, 64), J)
            executed = 15 * 2.0 * (ex_fwd if dom == "dense_fwd" else ex_rev)
            ex_t = executed / (per_eval[dom] * 1e-3) / 1e12
            return {"bound": "tensor", "achieved": achieved, "peak": pk_s / 15.0,
                    "unit": "TFLOP/s", "frac": achieved / (pk_s / 15.0),
                    "traffic": captured_traffic(kern, args.workload, J),
                    "kernel": kern + " (float-pair products as exact BF16 slice "
                                     "products on tcgen05)",
                    "peak_source": "derived: " + pk_src
                                   + " / 15 BF16 slice products per float-pair multiply-add",
                    "algorithmic_flops_per_launch": flops, "doublings": J,
                    "frac_of_bf16_peak": achieved / pk_s,
                    "executed_bf16_tflops": ex_t, "executed_frac": ex_t / pk_s}
        if mixed:
            return {"bound": "alu", "achieved": achieved, "peak": pair_peak,
                    "unit": "TFLOP/s", "frac": achieved / pair_peak,
                    "traffic": captured_traffic(kern + "<float2>", args.workload, J),
                    "kernel": kern + "<float2> (float-pair products on the FP32 pipes)",
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x "
                                   f"{sm_mhz:.0f} MHz / 12 FP32 instructions per "
                                   "float-pair multiply-add, 2 flops each",
                    "algorithmic_flops_per_launch": flops, "doublings": J}
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": None, "kernel": kern + "<double> (FP64 DFMA)",
                "peak_source": "nominal FP64 rate of a GB300",
                "algorithmic_flops_per_launch": flops, "doublings": J}

    # a grid pass: one multiply-add per (point, mu, nu) within r_c
    gflops = 2.0 * dims["sum_npt2"]

    def grid_roof_of(g):
        if not per_eval.get(g, 0.0) > 0.0:
            return None
        gach = gflops / (per_eval[g] * 1e-3) / 1e12
        if not mixed:
            return {"bound": "alu", "achieved": gach, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": gach / FP64_PEAK_TFLOPS, "traffic": None,
                    "kernel": f"{g}_fp64 (FP64 DFMA)",
                    "peak_source": "nominal FP64 rate of a GB300"}
        nu = solver.get_array("tile_nu_tc").astype(np.int64)  # functions per 128-point tile
        if g == "vmat":  # 8 slice products per 16-point K step of a V group (runs of
            # consecutive tiles), M = 128 rows, N = the group's union list padded to 16
            t0v = solver.get_array("vgroup_t0").astype(np.int64)
            gnu = solver.get_array("vgroup_nu").astype(np.int64)
            npad = np.maximum(16, ((gnu + 15) // 16) * 16)
            executed = float((8 * 2.0 * 128 * npad * 128 * np.diff(t0v)).sum())
        else:  # 9 slice products per 16-function K step, N = occupied orbitals padded to 32
            nmpad = sum(max(32, ((min(128, N - m0) + 31) // 32) * 32) for m0 in range(0, N, 128))
            ksteps = np.maximum(1, (nu + 15) // 16)
            executed = float((9 * 2.0 * 128 * nmpad * 16 * ksteps).sum())
        return {"bound": "tensor", "achieved": gach, "peak": pk_s, "unit": "TFLOP/s",
                "frac": gach / pk_s,
                "traffic": captured_traffic(f"{g}_tc_kernel", args.workload),
                "kernel": f"{g}_tc_kernel", "peak_source": pk_src,
                "algorithmic_flops_per_launch": gflops,
                "executed_tflops": executed / (per_eval[g] * 1e-3) / 1e12,
                "executed_frac": executed / (per_eval[g] * 1e-3) / 1e12 / pk_s}

    passes = {g: grid_roof_of(g) for g in ("rho", "vmat")}
    passes.update({d: dense_roof(d) for d in ("dense_fwd", "dense_rev")})
    # the dominant kernel is the stage with the largest time
    dom = max((k for k in passes if passes[k] is not None), key=lambda k: per_eval[k])
    roof = passes[dom]
    gdom = max((k for k in ("rho", "vmat") if passes[k] is not None), key=lambda k: per_eval[k])
    grid_roof = passes[gdom]

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32+bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": args.precision,
                   "parallelism": f"replicas{world}",
                   "l2": ("inputs larger than L2 (resident basis slices and grids), "
                          "steps back to back in one minimization" if large else
                          "flushed (512 MB write) before every timed step"),
                   "evals_timed": int(all_evals), "E_last": E_last,
                   "stage_ms_per_eval": per_eval,
                   "M": M, "N": N, "grid_points": dims["G"],
                   "sum_npt2": dims["sum_npt2"], "fp64_path": fp64,
                   "E_run_Ha": E_run},
        "roofline": roof,
        "roofline_grid": grid_roof,
        "roofline_passes": passes,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(d, WORKLOADS[args.workload], args.workload)
    print(json.dumps(line))


def run_batch(args):
    """The batched workload: K L-BFGS steps of one batched minimization of all
    molecules (each with its own line search), timed back to back; value =
    molecule energy+gradient evaluations per second.  The plain FP64 path runs
    each molecule's own launch sequence."""
    import torch

    from paper_2101_12597_gb300 import build as b
    from paper_2101_12597_gb300.etdm import ETDMBatch

    world, rank, local = dist_setup(args.gpus)
    b.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    mols = workload_system(args.workload)
    n = len(mols)
    t_setup = time.perf_counter()
    bt = ETDMBatch(mols, precision="mixed", device=local)
    t_setup = time.perf_counter() - t_setup
    a0 = torch.tensor(bt.pack([d["a0"] for d in mols]), device=dev)
    dims_M = [m.M for m in bt.systems]
    if args.profile_once:
        bt.energy_grad(a0)
        torch.cuda.synchronize()
        bt.check()
        print(json.dumps({"profile_once": True, "workload": args.workload}))
        return
    # warm-up, then the timed minimization from the start point
    a = a0.clone()
    if args.warmup:
        bt.minimize(a, args.warmup)
    torch.cuda.synchronize()
    bt.lbfgs_reset()
    a = a0.clone()
    bt.launches()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    barrier(world)
    torch.cuda.synchronize()
    ev0.record()
    E_h, al_h, tr_h = bt.minimize(a, args.steps)
    ev1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = bt.launches()
    total_ms = ev0.elapsed_time(ev1)
    evals = int(tr_h.sum())
    t_max = reduce_max(total_ms, world, dev)
    all_evals = reduce_sum(evals, world, dev)
    value = all_evals / (t_max / 1e3)

    # one batched evaluation (graph) at the start point, and its stages timed
    # one by one (the same kernels launched outside the graph)
    Eb, _ = bt.energy_grad(a0)
    torch.cuda.synchronize()
    reps = 10
    ev0.record()
    for _ in range(reps):
        bt.energy_grad(a0)
    ev1.record()
    torch.cuda.synchronize()
    graph_ms = ev0.elapsed_time(ev1) / reps
    bt.lib.etdm_set_profiling(bt.h, 1)
    bt.launches()
    for _ in range(3):
        bt.energy_grad(a0)
    torch.cuda.synchronize()
    ms = np.zeros(8)
    cnt = np.zeros(8, dtype=np.int64)
    import ctypes
    bt.lib.etdm_stage_times(bt.h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    bt.lib.etdm_set_profiling(bt.h, 0)
    names = ["dense_fwd", "rho", "potential", "vmat", "dense_rev"]
    stage = {k: float(ms[i] / max(1, cnt[i])) for i, k in enumerate(names)}

    # end to end through the host-buffer entry point
    a_host = bt.pack([d["a0"] for d in mols])
    bt.energy_grad_host(a_host)
    n_e2e = 10
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        E_run, _ = bt.energy_grad_host(a_host)
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * n * n_e2e / e2e_dt, "unit": "evals/s",
           "h2d_bytes_per_step": 8 * bt.nvar, "d2h_bytes_per_step": 8 * (bt.nvar + n),
           "evals": n * n_e2e}

    # the plain FP64 path: every molecule on its own launch sequence
    fp64 = None
    if not args.no_fp64_compare:
        ref = ETDMBatch(mols, precision="fp64", device=local)
        E64, _ = ref.energy_grad_host(a_host)
        torch.cuda.synchronize()
        k64 = 3
        ev0.record()
        for _ in range(k64):
            ref.energy_grad(a0)
        ev1.record()
        torch.cuda.synchronize()
        fp64 = {"value": n * k64 / (ev0.elapsed_time(ev1) / 1e3), "unit": "evals/s",
                "evals_timed": n * k64, "dE_Ha_max": float(np.abs(E_run - E64).max()),
                "launches_per_batch_eval": None}
        ref.launches()
        ref.energy_grad(a0)
        torch.cuda.synchronize()
        fp64["launches_per_batch_eval"] = ref.launches()
        ref.close()

    # roofline of the dominant stage of the batched evaluation
    peaks, src = measured_peaks()
    layout = (ctypes.c_int64 * 12)()
    bt.lib.etdm_layout(bt.h, layout)
    sum_npt2 = int(layout[10])
    dom = max(stage, key=lambda k: stage[k])
    pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", BF16_FALLBACK_TFLOPS))
    if dom in ("rho", "vmat"):
        ach = 2.0 * sum_npt2 / (stage[dom] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": captured_traffic(f"{dom}_tc_kernel", args.workload),
                "kernel": f"{dom}_tc_kernel (all molecules in one launch)",
                "peak_source": f"{src} dense bf16 (sustained)"}
    elif dom == "potential":
        # the five half-spectrum passes: each reads and writes the half spectrum
        # (float-pair complex, 16 B) once; the first reads rho, the last v_ext and
        # rho and writes v (FP64), v dV (pairs): bytes per grid point
        G = int(layout[3])
        nbytes = G * (2 * 5 * 16 * 0.5 + 8 + 3 * 8 + 8 + 8)
        ach = nbytes / (stage[dom] * 1e-3) / 1e9
        hbm = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None,
                "kernel": "potential passes (zfwd, yfft x2, xpois, zinv_pot) over all molecules",
                "peak_source": f"{src} copy bandwidth"}
    else:
        macs = 0.0
        for m in bt.systems:
            J = int(m.get_array("doublings")[0])
            f_, r_ = dense_macs(m.M, m.N, m.V, J)
            macs += f_ if dom == "dense_fwd" else r_
        ach = 2.0 * macs / (stage[dom] * 1e-3) / 1e12
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        pair_peak = 152 * 128 * sm_mhz * 1e6 * 2.0 / 12.0 / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": pair_peak, "unit": "TFLOP/s",
                "frac": ach / pair_peak, "traffic": None,
                "kernel": f"{dom} batched float-pair chains (one block per molecule)",
                "peak_source": "derived float-pair multiply-add rate of the FP32 pipes"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "mixed",
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (resident basis slices and grids of 148 "
                         "molecules), steps back to back in one batched minimization",
                   "molecules": n, "M_range": [min(dims_M), max(dims_M)],
                   "evals_timed": int(all_evals),
                   "batched_eval_graph_ms": graph_ms,
                   "molecule_evals_per_s_graph": n / (graph_ms * 1e-3),
                   "stage_ms_per_batched_eval": stage, "setup_s": t_setup,
                   "autotuner": {"tiles_per_v_group": bt.tune()[0],
                                 "ms_per_batched_eval_by_tiles": bt.tune()[1]},
                   "fp64_path": fp64, "E_sum_Ha": float(np.sum(E_run))},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        from oracle.etdm_oracle import Oracle
        pick = list(range(0, n, 15))
        t = 0.0
        for i in pick:
            o = Oracle(mols[i])
            o.reference()
            t0 = time.perf_counter()
            o.energy_grad(mols[i]["a0"])
            t += time.perf_counter() - t0
        line["cpu_baseline"] = {
            "value": len(pick) / t, "unit": "evals/s", "cores": oracle_threads(),
            "kind": "oracle",
            "sample": f"oracle energy+gradient evaluations of {len(pick)} of the {n} molecules "
                      "(every 15th; set-up not timed)"}
    print(json.dumps(line))


def _kplane_sample(o, D, v, i):
    """Seconds the k-point oracle takes for one x-plane of one k-point's grid
    work: the Bloch basis on the plane (Eq. 5), the density there (Eq. 2) and
    the plane's part of the potential matrix (Eq. 11)."""
    per = int(o.n[1] * o.n[2])
    t0 = time.perf_counter()
    Xp = o.basis_plane_k(i, 0)
    np.einsum("pa,pa->p", Xp @ D, Xp.conj()).real
    Xp.conj().T @ (v[i * per:(i + 1) * per, None] * Xp)
    return time.perf_counter() - t0


KPLANE_SAMPLE = ("the k-point oracle's grid work (Bloch basis values, density, potential-"
                 "matrix part) on {k} of the {n} x-planes of one k-point of {w}, scaled by "
                 "{n}/{k} x {nk} k-points to one evaluation; the dense steps (eigendecomposition "
                 "of iA(k), M x M complex products) and the FFTs are left out")


def run_kpoints(args):
    """The full-A path (FP64): K L-BFGS steps of one minimization from A = 0,
    the reference built on the device (generalized eigenvectors of h_core(k),
    Fermi-Dirac occupations; for a workload without k-points the Gamma point
    with integer occupation)."""
    import torch
    from paper_2101_12597_gb300 import build as b
    from paper_2101_12597_gb300.etdm import ETDM

    world, rank, local = dist_setup(args.gpus)
    b.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    d = workload_system(args.workload)
    solver = ETDM(d, precision="fp64", device=local, expm=args.expm, ref_update=args.ref_update,
                  param="full")
    a0 = torch.zeros(solver.var_shape, dtype=torch.float64, device=dev)
    if args.profile_once:
        solver.energy_grad(torch.tensor(d["a0"], dtype=torch.float64, device=dev))
        torch.cuda.synchronize()
        solver.check()
        print(json.dumps({"profile_once": True, "workload": args.workload}))
        return
    a = a0.clone()
    if args.warmup:
        solver.minimize(a, args.warmup)
    torch.cuda.synchronize()
    solver.lbfgs_reset()
    a = a0.clone()
    solver.set_profiling(True)
    solver.stage_times()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0.record()
    E_h, al_h, tr_h = solver.minimize(a, args.steps)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = ev0.elapsed_time(ev1)
    stage_ms, stage_n, launches = solver.stage_times()
    solver.set_profiling(False)
    evals = int(tr_h.sum())
    t_max = reduce_max(total_ms, world, dev)
    all_evals = reduce_sum(evals, world, dev)
    value = all_evals / (t_max / 1e3)
    # end to end through the host-buffer entry point (at the workload's seeded
    # variables when they are full-A variables, else at A = 0)
    a_host = np.ascontiguousarray(d["a0"]) if np.size(d["a0"]) == solver.nvar \
        else np.zeros(solver.var_shape)
    solver.energy_grad_host(a_host)
    torch.cuda.synchronize()
    n_e2e = min(args.steps, 5)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        solver.energy_grad_host(a_host)
    e2e_dt = reduce_max(time.perf_counter() - t0, world, dev)
    e2e = {"value": world * n_e2e / e2e_dt, "unit": "evals/s",
           "h2d_bytes_per_step": 8 * solver.nvar, "d2h_bytes_per_step": 8 * solver.nvar + 8,
           "evals": n_e2e}
    per_eval = {k: v / max(evals, 1) for k, v in stage_ms.items()}
    # FP64 ALU bound: the complex products of the dense stages (9 per evaluation
    # on the eigendecomposition route: U, O, D, then H O, O^dag(HO), L W,
    # W^dag(LW), W X, X W^dag; 4 on the scaling-and-squaring route: O, D, H O,
    # O^dag(HO)), and the exp stage (eigensolver, or the products of the Taylor
    # polynomial and the squarings)
    M, nk = solver.M, solver.nvar // (solver.M * solver.M)
    zflop = 8.0 * M ** 3 * nk  # one batched complex product
    nprod = 9 if args.expm == "eig" else 4
    dense_ms = per_eval["dense_fwd"] + per_eval["dense_rev"]
    roof_dense = {"bound": "alu", "kernel": f"zgemm_kernel ({nprod} batched complex products "
                  "per evaluation in the dense stages)",
                  "achieved": nprod * zflop / (dense_ms * 1e-3) / 1e12,
                  "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "traffic": None,
                  "peak_source": "nominal FP64 rate of a GB300 (no measured FP64 figure)"}
    roof_dense["frac"] = roof_dense["achieved"] / roof_dense["peak"]
    if args.expm == "eig":
        # the eigensolver: Householder reduction (16/3 M^3 real flops per complex
        # matrix), QL with rotations applied to Z (about 3 M^3 for ~1.5 sweeps per
        # eigenvalue over M rows), back-transformation (8 M^3)
        eflop = (16.0 / 3.0 + 3.0 + 8.0) * M ** 3 * nk
        roof = {"bound": "alu", "kernel": "zhetrd_kernel + ztql_kernel + zback_kernel (the "
                "eigendecomposition of iA(k), Eq. 35)",
                "achieved": eflop / (per_eval["eig"] * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "traffic": None,
                "peak_source": "nominal FP64 rate of a GB300 (no measured FP64 figure)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:  # every step is a batched complex product (the exp stage's count varies with |A|)
        roof = dict(roof_dense)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "fp64",
                   "param": "full A(k)" + ("" if "kpts" in d else " at the Gamma point, integer "
                                           "occupation"),
                   "expm": ("eigendecomposition of iA(k) (Eq. 35), exact gradient (Eq. 39)"
                            if args.expm == "eig" else
                            "scaling and squaring (Eq. 38), approximate gradient (Eq. 42), "
                            f"reference updates {args.ref_update}"),
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (complex matrices of every k-point, grids), "
                         "steps back to back in one minimization",
                   "evals_timed": int(all_evals), "E_first": float(E_h[0]),
                   "E_last": float(E_h[-1]), "stage_ms_per_eval": per_eval,
                   "M": M, "n_k": nk},
        "roofline": roof, "roofline_dense": roof_dense, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        from oracle.etdm_kpoints import BlochOracle
        dk = d if "kpts" in d else dict(d, kpts=np.zeros((1, 3)), kw=np.ones(1), kT=0.0)
        o = BlochOracle(dk, cache_x=False)
        rng = np.random.default_rng(0)
        C = rng.normal(size=(o.M, o.M)) + 1j * rng.normal(size=(o.M, o.M))
        D = (C @ C.conj().T) / o.M
        v = rng.normal(size=o.G)
        t, k = 0.0, 0
        while k < int(o.n[0]) and (k == 0 or t < 10.0):
            t += _kplane_sample(o, D, v, k)
            k += 1
        n = int(o.n[0])
        line["cpu_baseline"] = {"value": 1.0 / (t / k * n * o.nk), "unit": "evals/s",
                                "cores": oracle_threads(), "kind": "oracle",
                                "sample": KPLANE_SAMPLE.format(k=k, n=n, nk=o.nk,
                                                               w=WORKLOADS[args.workload])}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="water576",
                    help="water576 (the largest workload on one GPU: the default), "
                         "water32, the 8-atom molecule, or the batch of 148 molecules")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--param", choices=["occvirt", "full"], default="occvirt",
                    help="full: the full-A path (FP64; at the Gamma point with integer "
                         "occupation for the water and molecule workloads), for the paper's "
                         "comparison of the occupied-virtual route with the full-A routes")
    ap.add_argument("--expm", choices=["eig", "ss"], default="eig",
                    help="crystal64: exp(A(k)) by the eigendecomposition of iA (Eq. 35, exact "
                         "gradient) or by scaling and squaring (Eq. 38, approximate gradient)")
    ap.add_argument("--ref-update", type=int, default=0,
                    help="crystal64 with --expm ss: reference update every n steps, -1 by "
                         "the |L| < 3 |[A, L]| test, 0 never")
    ap.add_argument("--profile-once", action="store_true",
                    help="set up, run one energy+gradient evaluation, exit (for ncu)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dense-tc", type=int, choices=[-1, 0, 1], default=0,
                    help="float-pair dense products on the tensor cores: 0 the large ones "
                         "(default), 1 all, -1 none")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "molecules148":
        run_batch(args)
    elif args.workload == "crystal64" or args.param == "full":
        run_kpoints(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
