"""Host-side logic of bench.py that runs without a GPU: the replica aggregation
over ranks (gloo, world size 2), the oracle arm launched under torchrun, and
the count of threads the oracle's timing reports."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _aggregate_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each replica times its own steps; value = all evaluations / slowest rank
        ms = [120.0, 180.0][rank]
        evals = [13, 11][rank]
        bench.barrier(world)
        t_max = bench.reduce_max(ms, world, "cpu")
        n_all = bench.reduce_sum(evals, world, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"t_max": t_max, "n_all": n_all,
                       "value": n_all / (t_max / 1e3)}, f)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_max_time_sum_of_evaluations(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_aggregate_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["t_max"] == 180.0
        assert r["n_all"] == 24.0
        assert r["value"] == pytest.approx(24 / 0.18)


def test_single_rank_helpers_need_no_process_group():
    assert bench.reduce_max(2.5, 1, "cpu") == 2.5
    assert bench.reduce_sum(7, 1, "cpu") == 7
    bench.barrier(1)


def test_reference_arm_under_torchrun_prints_one_line():
    """Two ranks of the oracle arm: rank 0 alone runs and prints; both exit 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "small", "--steps", "2", "--warmup", "1"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    ln = lines[0]
    assert ln["impl"] == "reference" and ln["n_gpus"] == 2 and ln["steps"] == 2
    assert ln["value"] > 0 and ln["e2e"]["value"] == ln["value"]
    assert ln["cpu_baseline"]["value"] == ln["value"]
    # torchrun sets OMP_NUM_THREADS=1 for its workers unless it is already set
    if "OMP_NUM_THREADS" not in os.environ and "OPENBLAS_NUM_THREADS" not in os.environ:
        assert ln["cpu_baseline"]["cores"] == 1


def test_oracle_threads_without_threadpoolctl(monkeypatch):
    monkeypatch.setitem(sys.modules, "threadpoolctl", None)  # import raises ImportError
    ncpu = len(os.sched_getaffinity(0))
    for k in ("OPENBLAS_NUM_THREADS", "GOTO_NUM_THREADS", "OMP_NUM_THREADS"):
        monkeypatch.delenv(k, raising=False)
    assert bench.oracle_threads() == ncpu
    monkeypatch.setenv("OMP_NUM_THREADS", "1")
    assert bench.oracle_threads() == 1
    monkeypatch.setenv("OPENBLAS_NUM_THREADS", str(ncpu + 5))  # takes precedence, capped
    assert bench.oracle_threads() == ncpu


def test_clock_record_parsing(tmp_path):
    """The sampler's CSV (nvidia-smi, no header, no units): median SM clock under
    load, the maximum, and every throttle reason seen active."""
    p = tmp_path / "clocks.csv"
    p.write_text(
        "0, 1965, 2070, 950.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, [N/A], 2070, [N/A], 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1995, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbled line\n")

    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

        def kill(self):
            pass

    c = bench.Clocks(0)
    c.proc, c.path = Proc(), str(p)
    r = c.stop()
    assert r == {"sm_mhz": 1995.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 4}
    assert not p.exists()
    p.write_text("0, 1410, 2070, 700.0, 0x0000000000000048, Active, Not Active, Active, Not Active\n")
    c.proc, c.path = Proc(), str(p)
    assert c.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi on the path
    monkeypatch.setattr(bench.tempfile, "tempdir", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None
    assert list(tmp_path.iterdir()) == []  # the temporary file is gone


def test_oracle_plane_sample_is_the_oracles_grid_work():
    """The bounded sample the CPU baseline takes of the 192^3 water box: one
    x-plane of the oracle's own density and potential-matrix code.  On a small
    system the per-plane pieces add up to the oracle's whole-grid results."""
    import numpy as np
    import etdm_synth as synth
    d = synth.config_small_molecule()
    o, D, v = bench._plane_sample_setup(d)
    assert bench._plane_sample(o, D, v, 3) > 0.0
    per = int(o.n[1] * o.n[2])
    rho = np.concatenate([o.density_plane(o.basis_plane(i), D) for i in range(int(o.n[0]))])
    np.testing.assert_allclose(rho, o.density(D).reshape(-1), rtol=1e-13, atol=1e-15)
    Vm = sum(o.potential_plane(o.basis_plane(i), v[i * per:(i + 1) * per])
             for i in range(int(o.n[0]))) * o.dV
    np.testing.assert_allclose(Vm, o.potential_matrix(v), rtol=1e-12, atol=1e-14)


def test_captured_traffic_matches_source_hash_and_doublings(tmp_path, monkeypatch):
    """The traffic of a kernel comes from a committed summary line only while
    the kernel's source is unchanged, and for the dense chains only at the
    doubling count it was captured with."""
    import hashlib
    src = tmp_path / "paper_2101_12597_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("// kernel source\n")
    h = hashlib.sha256((src / "k.cu").read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_w.md").write_text(
        "text before\n"
        f"traffic a_kernel 1000 k.cu:{h} w1\n"
        f"traffic b_kernel 2000 k.cu:{h} w1 doublings=3\n"
        f"traffic c_kernel 3000 k.cu:{'0' * 16} w1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.captured_traffic("a_kernel", "w1") == 1000
    assert bench.captured_traffic("a_kernel", "w1", 5) == 1000  # no count on the line
    assert bench.captured_traffic("a_kernel", "w2") is None
    assert bench.captured_traffic("b_kernel", "w1", 3) == 2000
    assert bench.captured_traffic("b_kernel", "w1", 4) is None
    assert bench.captured_traffic("c_kernel", "w1") is None  # source changed since


def test_l2_rule_per_workload_and_precision():
    """Steps run back to back only where a step's inputs exceed L2: the mixed
    path's resident slices from water32 up, the FP64 path's dense matrices from
    water216 up; every other run flushes L2 before each timed step."""
    assert bench.runs_back_to_back("water576", "mixed")
    assert bench.runs_back_to_back("water32", "mixed")
    assert not bench.runs_back_to_back("water32", "fp64")
    assert bench.runs_back_to_back("water216", "fp64")
    assert not bench.runs_back_to_back("small", "mixed")
