"""The N-GPU bench runs independent replicas (the solve has no data-parallel split):
per-rank seeds and the max-over-ranks time. The host side of that path, with two gloo
ranks on CPU (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed(7, rank)
    ms = 10.0 + 5.0 * rank                  # the slower rank decides the reported time
    out[rank] = (seed, bench.max_over_ranks(ms, world, device="cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == 7 and res[1][0] == 8           # distinct seeds per replica
    assert res[0][1] == res[1][1] == 15.0              # max over ranks on every rank


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.rank_seed(4, 0) == 4
