"""bench.py's multi-rank plumbing on CPU: two gloo ranks, max-over-ranks
timing and the whole-job aggregate (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, lr = bench.dist_env()
    t = 1.0 + rank            # rank 1 is the slow one
    bench.barrier()
    tmax = bench.reduce_max(t)
    value = bench.aggregate(1e6, tmax, ws)
    q.put((rank, ws, r, lr, tmax, value))
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, lr, tmax, value in out:
        assert ws == 2 and r == rank and lr == rank
        assert tmax == 2.0                     # max over ranks
        assert value == pytest.approx(1.0)     # 2 ranks x 1e6 updates / 2 s / 1e6


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.aggregate(2e6, 1.0, 1) == 2.0
