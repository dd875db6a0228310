"""The multi-GPU path of the benchmark is replicas only (the window does not shard on one node): each rank runs an
independent copy with its own noise key, and the whole-job rate is the units all ranks processed over the slowest
rank's time.  These tests run that host logic as two gloo ranks on the CPU (127.0.0.1)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = [120.0, 80.0][rank]
    secs = [2.0, 4.0][rank]
    rate = bench.whole_job_rate(units, secs, world, device="cpu")
    seed = bench.replica_seed(12345, rank)
    mx = bench._max_over_ranks(secs, world, device="cpu")
    bench._barrier(world)
    q.put((rank, rate, seed, mx))
    dist.destroy_process_group()


def _run(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_replicas_whole_job_rate_and_seeds():
    out = _run(2)
    for rank, rate, seed, mx in out:
        assert rate == pytest.approx((120.0 + 80.0) / 4.0)   # all ranks' units over the slowest rank's time
        assert mx == 4.0
        assert seed == 12345 + rank
    assert out[0][2] != out[1][2]                           # independent noise keys


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0
    assert bench.replica_seed(7, 0) == 7
