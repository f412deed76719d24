"""The multi-process path of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs an independent replica (no collective on the
data path): the timing is the maximum over ranks after a barrier, the value is
the units all ranks processed over that time, and the reference arm runs on
rank 0 alone while the other ranks exit 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup("gloo")
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.5 + rank, w)          # rank 1 is the slow one
    rate = bench.whole_job_rate(1000.0, w, slowest)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((r, w, slowest, rate))


def test_max_over_ranks_and_whole_job_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for _, w, slowest, rate in res:
        assert w == 2 and slowest == 2.5                     # the max, on every rank
        assert rate == pytest.approx(2 * 1000.0 / 2.5)       # all ranks' units / slowest time


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_under_torchrun_world_2():
    """`bench.py --impl reference` launched like the multi-GPU bench: rank 0
    prints one JSON line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["steps"] == 2
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


def test_traffic_record_only_for_the_captured_launch(tmp_path, monkeypatch):
    """The DRAM traffic of the timed launch is reported only when the committed
    capture took exactly that launch: the same kernel sources (hash), workload,
    first iteration and number of iterations; anything else reads as no
    measurement (null), never as another launch's bytes."""
    sys.path.insert(0, ROOT)
    import bench
    rec = {"workload": "rosenbrock_1048576x64", "source_sha": bench.kernel_source_sha(), "first_iteration": 6,
           "iterations": 20, "dram_bytes_per_launch": 123456789}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.measured_traffic("rosenbrock_1048576x64", 6, 20) == 123456789
    assert bench.measured_traffic("rosenbrock_1048576x64", 7, 20) is None      # another first iteration
    assert bench.measured_traffic("rosenbrock_1048576x64", 6, 1) is None       # another launch form
    assert bench.measured_traffic("rastrigin_65536x128", 6, 20) is None        # another workload
    path.write_text(json.dumps(dict(rec, source_sha="0" * 16)))
    assert bench.measured_traffic("rosenbrock_1048576x64", 6, 20) is None      # sources changed since
    path.write_text("not json")
    assert bench.measured_traffic("rosenbrock_1048576x64", 6, 20) is None


def test_committed_traffic_record_matches_the_sources():
    """The committed record is the capture of the current kernel sources, for
    the timed launch of the default command (--steps 20 --warmup 5)."""
    sys.path.insert(0, ROOT)
    import bench
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.load(f)
    assert rec["source_sha"] == bench.kernel_source_sha()
    assert (rec["first_iteration"], rec["iterations"]) == (6, 20)
    assert bench.measured_traffic(rec["workload"], 6, 20) == rec["dram_bytes_per_launch"]
