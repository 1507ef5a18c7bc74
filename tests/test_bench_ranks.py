"""The multi-rank path of bench.py on CPU: world_size 2 over gloo (each rank
an independent replica; the job's time is the slowest rank's, its work the
sum over ranks), and the rank/world parsing of the launcher environment."""
import os
import socket

import pytest

import __graft_entry__  # noqa: F401
import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    t, n = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist)
    out.put((r, ws, local, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_over_gloo():
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
    assert [(r, ws, lr) for r, ws, lr, _, _ in res] == [(0, 2, 0), (1, 2, 1)]
    # every rank sees the slowest time and the summed work
    assert all(t == 20.0 and n == 3000 for _, _, _, t, n in res)


def test_single_process_reduction_is_the_identity(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.reduce_over_ranks(12.5, 77) == (12.5, 77)
