"""The multi-process replica path of bench.py on the CPU (gloo, world size 2):
every rank gets the slowest rank's time, and the whole-job rate counts every
rank's units over that time.  (On GPUs the same functions run over NCCL with
one process per GPU; each rank projects its own replica, no data exchange.)"""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], dist, device="cpu")
    out.put((rank, ms, bench.job_throughput(world, 1000, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [120.0, 80.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 120.0
        assert rate == pytest.approx(2 * 1000 / 0.12)


def test_single_process_paths():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.job_throughput(1, 500, 250.0) == pytest.approx(2000.0)


def test_cpu_baseline_both_oracles():
    """The CPU baseline leg (and the reference arm) times the oracle walker by
    default and the brute-force clipper on request; both run on a small case."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    w = W.config1(n_cells=4, det=16, pitch=0.3, nangles=4)
    for kind in ("walker", "clipper"):
        rate, threads, dt, n = bench.cpu_baseline(w, 64, kind=kind)
        assert n == 64 and rate > 0 and dt > 0 and threads >= 1
        assert "oracle walker" in bench.cpu_sample_text("walker", 64, w.geom.nrays)


def test_reference_arm_json_line():
    """`bench.py --impl reference` prints one JSON line with the contract's keys
    (run on a small workload, as on the host of a GPU machine)."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "kuhn24", "--steps", "1", "--warmup", "1",
                        "--cpu-sample", "256"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
