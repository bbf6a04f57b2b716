"""Multi-rank path of the bench on CPU (gloo, world size 2): every rank gets
its own share of the independent solves, the timed region's duration is the
maximum over ranks, and the value counts the work of all ranks."""
import os
import socket

import pytest

from paper_2107_01370_gb300 import replicas


def test_shard_covers_every_solve_once():
    for total in (1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s, c = replicas.shard(total, r, world)
                seen.extend(range(s, s + c))
            assert seen == list(range(total))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, count = replicas.shard(16, rank, world)
    local_seconds = 1.0 + rank               # rank 1 is the slower one
    t = replicas.max_over_ranks(local_seconds, dist)
    nodes = replicas.sum_over_ranks(count * 131072 * 10, dist)
    out.put((rank, start, count, t, replicas.aggregate_mlups(nodes, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    torch = pytest.importorskip("torch")
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
    assert [r[1:3] for r in res] == [(0, 8), (8, 8)]
    assert all(r[3] == 2.0 for r in res)
    assert all(abs(r[4] - 16 * 131072 * 10 / 2.0 / 1e6) < 1e-9 for r in res)
