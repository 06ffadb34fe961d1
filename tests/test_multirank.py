"""The N > 1 bench path on CPU with gloo: every rank runs an independent
replica, the step time is the max over ranks, and the reference arm runs on
rank 0 only (the other ranks exit 0 without work)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks(10.0 * rank + 5.0, world, "cpu")
    w, r, lr = bench.dist_env()

    class Args:
        steps, warmup = 1, 0
    rc = bench.run_reference(Args()) if rank != 0 else 0
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, (w, r, lr), rc))


def test_two_rank_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, got, env, rc in res:
        assert got == pytest.approx(15.0)          # max over ranks
        assert env == (world, rank, rank)
        assert rc == 0                               # non-zero ranks skip the reference arm
