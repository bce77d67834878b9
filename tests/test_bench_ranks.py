"""The benchmark's multi-rank logic on the CPU (gloo, world size 2): the job's
time is the slowest rank's, its throughput counts every rank's keys, and the
reference arm runs on rank 0 alone.  The sort itself has no exchange step (one
GPU per rank runs an independent replica), so these are the only cross-rank
operations."""
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench._max_over_ranks(1.5 + rank, torch.device("cpu"))
    q.put((rank, ms, bench._job_value(1 << 24, ws, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 2.5                                  # the slower rank's time on both ranks
        assert value == pytest.approx((1 << 24) * 2 / 2.5e-3 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import torch
    import bench
    assert bench._max_over_ranks(3.25, torch.device("cpu")) == 3.25
    assert bench._job_value(1000, 1, 1.0) == pytest.approx(1e-3)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
