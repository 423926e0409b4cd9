"""The multi-rank (torchrun) host logic of bench.py on CPU with the gloo backend,
world size 2: rendezvous, barrier, and the max over ranks of the elapsed time
that the whole-job number divides by.  Roots shard with no data-path
collective, so this is the only communication the bench does."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "BCTS_BENCH_BACKEND": "gloo"})
    import torch
    import torch.distributed as dist
    import bench
    w, r, lr = bench.dist_setup(world)
    bench.barrier(w)
    m = bench.max_over_ranks(w, 1.5 + r, torch.device("cpu"))
    q.put((r, w, lr, m))
    dist.destroy_process_group()


def test_two_rank_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 2 for g in got)
    assert all(g[3] == pytest.approx(2.5) for g in got)
