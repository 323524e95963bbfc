"""Multi-rank path of the benchmark on the CPU (gloo, world size 2).

The contact path shards by environment with no exchange step: each rank runs
its own scenes and only the timings are combined (slowest rank, total pairs).
This checks that combination and that ranks get distinct work, with two gloo
processes on 127.0.0.1.
"""

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


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: 10 + r ms, 1000 * (r + 1) pairs
    res = bench.combine_ranks(10.0 + rank, 1000 * (rank + 1), 1.0 + 2 * rank, 500 * (rank + 1),
                              world, torch.device("cpu"))
    dist.barrier()
    q.put((rank, res, bench.rank_scene_seeds(rank, 3)))
    dist.destroy_process_group()


def test_two_rank_combination_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, res, seeds in out:
        assert res == (11.0, 3000.0, 3.0, 1500.0)  # MAX of times, SUM of pairs
    assert not set(out[0][2]) & set(out[1][2])  # distinct scenes per rank


def test_single_rank_passthrough():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5, 7, 1.5, 3, 1, None) == (5.0, 7.0, 1.5, 3.0)
