"""The multi-rank path of bench.py (one independent channel per rank, no
collective on the data path) on CPU: world_size-2 gloo process groups check
the max-over-ranks timing, the whole-job aggregate and the sharding of an
ensemble's channels over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank timed its own replica; the job time is the slowest rank's
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    value = bench.aggregate_rate(1000, 50, ms * 1e-3, world)
    mine = bench.shard(range(64), rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.barrier()
    out.put((rank, ms, value, got))
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, got in res:
        assert ms == 15.0                              # max over ranks
        assert value == pytest.approx(2 * 1000 * 50 / 0.015)
        flat = sorted(x for part in got for x in part)
        assert flat == list(range(64))                 # every channel exactly once
        assert not set(got[0]) & set(got[1])


def test_single_process_helpers():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
    assert bench.aggregate_rate(10, 2, 0.5, 1) == 40.0
