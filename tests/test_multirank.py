"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
solves its own seeded problem set (weak scaling, no collective on the data
path) and the job's time is the slowest rank's (max over ranks)."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    probs = bench._problems(16, rank, 9)
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    mine = [(p.alpha, p.beta, float(p.coeffs.sum()), float(p.yU[0].sum())) for p in probs]
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, everyone))


def test_two_ranks_disjoint_problems_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, everyone in out:
        assert slowest == 20.0                       # max over ranks, on every rank
        r0, r1 = everyone
        assert [x[:2] for x in r0] == [x[:2] for x in r1]   # same (alpha, beta) grid
        assert all(a[2:] != b[2:] for a, b in zip(r0, r1))  # different seeded inputs
