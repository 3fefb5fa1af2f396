"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): one
replica per rank, whole-job time = slowest rank, work = sum over ranks, and
every replica draws its own input stream."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, ev, e2e, e2e_ev = bench.combine_ranks(10.0 + rank, 1000.0 * (rank + 1), 0.5 * (rank + 1), 7.0,
                                              world, torch.device("cpu"))
    out[rank] = (ms, ev, e2e, e2e_ev, bench.replica_seed(123, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        ms, ev, e2e, e2e_ev, seed = res[r]
        assert ms == 11.0 and ev == 3000.0 and e2e == 1.0 and e2e_ev == 14.0
    assert res[0][4] != res[1][4]


def test_single_rank_passthrough():
    import bench
    assert bench.combine_ranks(3.0, 4.0, 5.0, 6.0, 1, None) == (3.0, 4.0, 5.0, 6.0)
