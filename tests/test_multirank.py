"""Multi-rank host logic of bench.py (weak scaling: every rank runs its own
workload, only a barrier and a max-of-times cross ranks), with world size 2
on the gloo backend on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench.dist_env()
    times = [0.5 + rank, 0.25]            # rank 1 is the slow one
    value, t = bench.aggregate(times, 1000, 2, ws)
    bench.barrier(ws)
    q.put((r, ws, value, t))
    dist.destroy_process_group()


def test_two_ranks_take_max_time_and_sum_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, value, t in out:
        assert ws == 2
        assert t == pytest.approx(1.75)               # max over ranks of 0.75 / 1.75
        assert value == pytest.approx(1000 * 2 * 2 / 1.75)


def test_pairs_per_step_counts_every_level():
    import bench
    # 200k objects in 40 segments of 5000 -> 2560 centroids -> one top segment
    assert bench.pairs_per_step(200000, 64, 5000, 10) == 200000 * 64 * 10 + 2560 * 64 * 10
    assert bench.pairs_per_step(100, 8, 1000, 3) == 100 * 8 * 3
    # 1000 objects -> 10 segments -> 100 centroids, which fit one segment
    assert bench.pairs_per_step(1000, 10, 100, 0) == 1000 * 10 + 100 * 10
