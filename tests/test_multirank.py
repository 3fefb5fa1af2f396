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


# ---------------------------------------------------------------------------
# Shards of the independent workloads (paper_2305_02510_gb300/shard.py) on two
# gloo ranks, with the CPU oracle standing in for each rank's GPU.

def test_partitions_cover_every_unit_once():
    import numpy as np
    from paper_2305_02510_gb300 import shard, workloads as W
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 5, 8, 64):
        for work in (rng.random(37), np.ones(4096), np.zeros(10), rng.integers(0, 5, 100).astype(float),
                     np.array([1e6] + [1.0] * 30)):
            b = shard.contiguous_split(work, world)
            assert b[0] == 0 and b[-1] == len(work) and np.all(np.diff(b) >= 0)
        total = rng.random(4096)
        b = shard.contiguous_split(total, world)
        share = np.array([total[b[r]:b[r + 1]].sum() for r in range(world)])
        assert share.max() <= total.sum() / world + total.max() + 1e-9
    for world in (1, 2, 3, 4):
        got = [shard.train_shard(512, r, world) for r in range(world)]
        assert sum(c for _, c in got) == 512 and all(c % 128 == 0 for _, c in got)
        assert all(got[r][0] + got[r][1] == got[r + 1][0] for r in range(world - 1))
        got = [shard.batch_shard(128, r, world, align=8) for r in range(world)]
        assert sum(c for _, c in got) == 128 and all(c % 8 == 0 for _, c in got)
    nets = W.batched_nets(count=30, steps=5, nmax=300)
    seen = []
    for r in range(3):
        first, mine = shard.network_shard(nets, r, 3)
        seen += [w["net_index"] for w in mine]
        assert all(w["net_index"] == first + k for k, w in enumerate(mine))
    assert seen == list(range(30))


def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch
    from oracle import bptt_ref as R, oracle as O
    from paper_2305_02510_gb300 import shard, workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # batched networks: this rank's contiguous range, streams keyed by global index
    nets = W.batched_nets(count=10, steps=30, nmax=200)
    first, mine = shard.network_shard(nets, rank, world)
    mine_r = {}
    for k, wl in enumerate(mine):
        st, raster, _ = O.run(wl, O.F32, 30, net_index=first + k)
        mine_r[first + k] = (raster, st.v)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine_r)
    # shared network: this rank's trains
    wl = W.shared_dense_i8(n=64, batch=8, steps=25)
    t0, cnt = shard.train_shard(8, rank, world, align=2)
    trains = {t0 + k: O.run(wl, O.INT, 25, net_index=t0 + k)[1] for k in range(cnt)}
    tg = [None] * world
    dist.all_gather_object(tg, trains)
    # BPTT data parallel: this rank's samples, loss scaled by its share
    task = W.bptt_task(batch=6, sizes=(12, 10, 4), steps=15, seed=3)
    task["w"] = [w * 2.0 for w in task["w"]]
    s0, sc = shard.batch_shard(6, rank, world)
    _, _, grads = R.gradients(shard.task_slice(task, s0, sc))
    grads = [g * (sc / task["batch"]) for g in grads]
    shard.allreduce_gradients(grads)
    if rank == 0:
        out["batched"] = {k: v for g in gathered for k, v in g.items()}
        out["trains"] = {k: v for g in tg for k, v in g.items()}
        out["grads"] = [g.numpy() for g in grads]
    dist.barrier()
    dist.destroy_process_group()


def test_shards_on_two_gloo_ranks_equal_one_rank():
    """Batched networks and shared-network trains split over two ranks, each
    rank running the oracle on its own share with global stream indices:
    every network and train appears exactly once and equals the single-rank
    run.  BPTT data parallel: the all-reduced gradients of the two batch
    shards equal the gradient of the whole batch."""
    import numpy as np
    from oracle import bptt_ref as R, oracle as O
    from paper_2305_02510_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    nets = W.batched_nets(count=10, steps=30, nmax=200)
    assert sorted(res["batched"]) == list(range(10))
    for b, wl in enumerate(nets):
        st, raster, _ = O.run(wl, O.F32, 30, net_index=b)
        assert np.array_equal(res["batched"][b][0], raster) and np.array_equal(res["batched"][b][1], st.v)
    wl = W.shared_dense_i8(n=64, batch=8, steps=25)
    assert sorted(res["trains"]) == list(range(8))
    for b in range(8):
        assert np.array_equal(res["trains"][b], O.run(wl, O.INT, 25, net_index=b)[1])
    task = W.bptt_task(batch=6, sizes=(12, 10, 4), steps=15, seed=3)
    task["w"] = [w * 2.0 for w in task["w"]]
    _, _, full = R.gradients(task)
    for a, b in zip(res["grads"], full):
        b = b.numpy()
        assert np.abs(b).max() > 0
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(b).max())


def _network_shard_rank(rank, world, port, out):
    """One rank of a sharded network with the oracle standing in for its GPU:
    each step it advances the whole oracle network from its own rows (the
    other ranks' rows of the current exchange window still zero) and keeps
    only its own neurons; the rows move through shard.exchange_loop, the
    product's exchange schedule, with a gloo all-reduce."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2305_02510_gb300 import shard, workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _sharded_workload()
    n, D, T = wl["n"], wl["max_delay"], wl["steps"]
    first, count = shard.neuron_shard(n, rank, world)
    mine = slice(first, first + count)
    words = (n + 31) // 32
    loc = np.zeros((T, n), np.uint8)          # rows this rank knows
    v = np.asarray(np.float32(wl["reset"]), np.float64).copy()
    r = np.zeros(n, np.int32)
    state = {"t": 0}

    def run(k):
        for u in range(state["t"], state["t"] + k):
            hist = np.zeros((D, n), np.uint8)
            for q in range(D):
                tau = u - D + q
                if tau >= 0:
                    hist[q] = loc[tau]
            st = O.state_from(wl, u, v, r, hist)
            st, row, _ = O.run(wl, O.F32, 1, state=st)
            v[mine], r[mine] = st.v[mine], st.r[mine]
            loc[u, mine] = row[0, mine]
        state["t"] += k

    def own_rows(t0, t1):
        bits = np.zeros((t1 - t0, words * 32), np.uint8)
        bits[:, mine] = loc[t0:t1, mine]
        return np.packbits(bits, axis=1, bitorder="little").view(np.uint32)

    def combine(rows):
        x = torch.from_numpy(rows.view(np.int32).astype(np.int64))
        dist.all_reduce(x, op=dist.ReduceOp.SUM)
        return x.numpy().astype(np.uint32)

    def put(t0, t1, rows):
        full = np.unpackbits(rows.view(np.uint8), axis=1, bitorder="little")[:, :n]
        loc[t0:t1] = full

    k = int(np.min(wl["delay"]))
    shard.exchange_loop(T, k, run, own_rows, combine, put)
    states = [None] * world
    dist.all_gather_object(states, (first, count, v[mine].copy(), r[mine].copy()))
    if rank == 0:
        out["raster"] = loc.copy()
        out["states"] = states
    dist.barrier()
    dist.destroy_process_group()


def _sharded_workload():
    import numpy as np
    from paper_2305_02510_gb300 import workloads as W
    wl = W.random_small(31, n=150, integer=False, steps=60, max_delay=5, p=0.06, events_rate=2.0)
    wl["delay"] = np.maximum(np.asarray(wl["delay"], np.int32), 2)
    return wl


def test_network_shards_on_two_gloo_ranks_equal_one_rank():
    """A single network split over two ranks by neuron range, exchanging spike
    rows every d_min = 2 steps: the combined raster and every neuron's state
    equal the unsharded oracle run (float32 mirror) bit for bit."""
    import numpy as np
    from oracle import oracle as O
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_network_shard_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    wl = _sharded_workload()
    st, want, _ = O.run(wl, O.F32, wl["steps"])
    assert want.sum() > 0 and np.array_equal(res["raster"], want)
    for first, count, v, r in res["states"]:
        assert np.array_equal(v, st.v[first:first + count]) and np.array_equal(r, st.r[first:first + count])
