"""Multi-rank host logic of bench.py, on CPU with gloo (world size 2).

Decodes shard by problem, so ranks exchange nothing on the data path; the
only collective is the timing reduction: every rank learns the slowest
rank's time, and the job's throughput is all ranks' units over that time."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [1.0 + rank, 10.0 - rank, 0.5 * (rank + 1)]
    got = bench.slowest_over_ranks(mine, dist)
    out.put((rank, got, bench.job_rate(30, world, got[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_reduction_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [2.0, 10.0, 1.0]          # max over the two ranks
        assert rate == pytest.approx(2 * 30 / 2.0)


def test_local_values_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_over_ranks([3, 4.5]) == [3.0, 4.5]
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_under_torchrun_prints_once():
    """--impl reference under torchrun with 2 ranks: rank 0 alone runs the
    oracle and prints one JSON line; the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "small", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
