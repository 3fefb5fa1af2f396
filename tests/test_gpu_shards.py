"""Shards of the independent workloads, each in its own context on one GPU,
against the context holding the whole family.

A rank of a multi-GPU run holds one contiguous range of the batched networks
(balanced by work) or of the shared network's input trains, with the Poisson
streams keyed by global index (sn_set_poisson_stream).  Whichever GPU runs a
shard, its networks and trains must then follow exactly the trajectories they
follow in one context: the shards' rasters and states, put together in order,
equal the whole context's bit for bit.  Every run here has one GPU, so the
shards run one after another on it; no shard waits on another."""

import numpy as np
import pytest

from oracle import compare
from paper_2305_02510_gb300 import shard, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def batch_run(nets, steps, first=0):
    from paper_2305_02510_gb300 import sn as S
    ctx = S.from_batch_workloads(nets, record_steps=steps, first=first)
    S.sn_run(ctx, steps)
    S.sn_sync(ctx)
    rasters = S.split_batch_raster(S.sn_get_spikes(ctx, 0, steps), ctx.net_n)
    v, r = S.sn_get_state(ctx)
    return rasters, v, r


@pytest.mark.parametrize("world", [2, 3, 8])
def test_batched_shards_equal_whole_family(world):
    steps = 120
    nets = W.batched_nets(count=48, steps=steps, nmax=1024)
    whole, v, r = batch_run(nets, steps)
    got, gv, gr, seen = [], [], [], 0
    for rank in range(world):
        first, mine = shard.network_shard(nets, rank, world)
        assert first == seen
        seen += len(mine)
        if not mine:
            continue
        rs, vv, rr = batch_run(mine, steps, first=first)
        got += rs
        gv.append(vv)
        gr.append(rr)
    assert seen == len(nets)
    for b in range(len(nets)):
        assert np.array_equal(got[b], whole[b]), f"network {b}"
    assert np.array_equal(np.concatenate(gv), v) and np.array_equal(np.concatenate(gr), r)
    # and the family against the oracle, at the first network of each shard
    off = np.cumsum([0] + [w["n"] for w in nets])
    for b in sorted({min(shard.network_shard(nets, q, world)[0], len(nets) - 1) for q in range(world)}):
        compare.check_float_run(nets[b], whole[b], v[off[b]:off[b + 1]], r[off[b]:off[b + 1]], steps,
                                net_index=b)


def test_generated_shard_equals_slice_of_family():
    """A rank can generate only its own networks (workloads.batched_nets with
    `first`): they are the same networks as in the whole family."""
    nets = W.batched_nets(count=20, steps=10, nmax=512)
    first, mine = shard.network_shard(nets, 1, 2)
    own = W.batched_nets(count=len(mine), first=first, steps=10, nmax=512)
    for a, b in zip(mine, own):
        assert a["n"] == b["n"] and np.array_equal(a["pre"], b["pre"]) and np.array_equal(a["weight"], b["weight"])


@pytest.mark.parametrize("world", [2, 4])
def test_shared_train_shards_equal_whole(world):
    from paper_2305_02510_gb300 import sn as S
    n, B, T = 256, 512, 40
    wl = W.shared_dense_i8(n=n, batch=B, steps=T)

    def run(first, count):
        ctx = S.from_shared_workload(wl, record_steps=T, first_train=first, trains=count)
        S.sn_run(ctx, T)
        bits = S.sn_get_spikes(ctx, 0, T)
        v, r = S.sn_get_state(ctx)
        return bits, v.reshape(count, n), r.reshape(count, n)

    bits, v, r = run(0, B)
    w = n // 32
    covered = 0
    for rank in range(world):
        first, count = shard.train_shard(B, rank, world)
        covered += count
        sb, sv, sr = run(first, count)
        assert np.array_equal(sb, bits[:, first * w:(first + count) * w])
        assert np.array_equal(sv, v[first:first + count]) and np.array_equal(sr, r[first:first + count])
    assert covered == B and bits.any()


def test_bptt_batch_shards_sum_to_whole_batch_gradient():
    """Data-parallel BPTT: two shards of 64 samples of the 700-1024-1024-20
    step, each through its own context with the loss scaled by its share;
    the summed gradients (what the all-reduce of a two-GPU run adds) equal
    the gradient of the whole 128-sample batch within the gradient tolerance
    (only the order of the weight gradient's sum over samples differs)."""
    from paper_2305_02510_gb300 import bptt
    dev = torch.device("cuda")
    task = W.bptt_task(steps=40)
    ws = [torch.tensor(w, device=dev, requires_grad=True) for w in task["w"]]

    def shard_grads(first, count):
        t = shard.task_slice(task, first, count)
        net = bptt.FFNet.from_task(t)
        for w in ws:
            w.grad = None
        counts = bptt.SNNFunction.apply(net, torch.tensor(t["input"], device=dev), *ws)
        loss = torch.nn.functional.cross_entropy(counts, torch.tensor(t["labels"], device=dev))
        return [g.clone() for g in shard.data_parallel_backward(loss, ws, count, task["batch"])]

    whole = shard_grads(0, 128)
    parts = [shard_grads(*shard.batch_shard(128, r, 2, align=8)) for r in range(2)]
    for l, g in enumerate(whole):
        s = parts[0][l] + parts[1][l]
        rel = float((s - g).norm() / g.norm())
        assert g.norm() > 0 and rel < 1e-5, (l, rel)


# ---------------------------------------------------------------------------
# One network over several GPUs: shard contexts (sn_create_shard), emulated
# here one after another on one GPU with the rows exchanged on the host, must
# reproduce the single pull context bit for bit.

def run_network_shards(wl, world, steps, flags=0):
    from paper_2305_02510_gb300 import sn as S
    ctxs = [S.from_workload_shard(wl, *shard.neuron_shard(wl["n"], r, world), record_steps=steps, flags=flags)
            for r in range(world)]
    k = S.sn_shard_info(ctxs[0])[2]
    ranges = [shard.neuron_shard(wl["n"], r, world) for r in range(world)]

    def run(n_steps):
        for c in ctxs:
            S.sn_run(c, n_steps)

    def own_rows(t0, t1):
        rows = []
        for c, (f, cnt) in zip(ctxs, ranges):
            full = S.sn_get_spikes(c, t0, t1)
            own = np.zeros_like(full)
            own[:, f // 32:(f + cnt + 31) // 32] = full[:, f // 32:(f + cnt + 31) // 32]
            rows.append(own)
        return rows

    def combine(rows):
        return np.sum([r.astype(np.uint64) for r in rows], axis=0).astype(np.uint32)

    def put(t0, t1, rows):
        for c in ctxs:
            S.sn_shard_put_spikes(c, t0, t1, rows)

    assert shard.exchange_loop(steps, k, run, own_rows, combine, put) == steps
    raster = S.unpack_raster(S.sn_get_spikes(ctxs[0], 0, steps), wl["n"])
    v = np.zeros(wl["n"], np.float32 if wl["dtype"] == "f32" else np.int32)
    r = np.zeros(wl["n"], np.int32)
    spikes = events = 0
    for c, (f, cnt) in zip(ctxs, ranges):
        vv, rr = S.sn_get_state(c)
        v[f:f + cnt], r[f:f + cnt] = vv[f:f + cnt], rr[f:f + cnt]
        _, sp, ev = S.sn_get_counters(c)
        spikes, events = spikes + sp, events + ev
        assert np.array_equal(S.unpack_raster(S.sn_get_spikes(c, 0, steps), wl["n"]), raster)
    return raster, v, r, spikes, events, k


@pytest.mark.parametrize("case,world,form", [("small-d2", 2, 0), ("small-d2", 3, 0x2000), ("sparse-float", 2, 0),
                                             ("sparse-float", 4, 0), ("sparse-float", 3, 0x2000),
                                             ("sparse-int", 3, 0)])
def test_network_shards_equal_single_context(case, world, form):
    """form 0x2000 (SN_PULL_CODED): the shards hold the coded pull store, the
    single context the plain one; the runs must still agree bit for bit."""
    from paper_2305_02510_gb300 import sn as S
    if case == "small-d2":
        wl = W.random_small(21, n=300, integer=False, steps=120, max_delay=5, p=0.05, events_rate=2.0)
        wl["delay"] = np.maximum(np.asarray(wl["delay"], np.int32), 2)   # smallest delay 2: exchange every 2 steps
        steps = 120
    else:
        wl = W.large_sparse(integer=case == "sparse-int", n=20_000, steps=80)
        steps = 80
    raster, v, r, spikes, events, k = run_network_shards(wl, world, steps, flags=form)
    assert k == int(np.min(wl["delay"]))
    whole = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=steps)
    S.sn_run(whole, steps)
    want = S.unpack_raster(S.sn_get_spikes(whole, 0, steps), wl["n"])
    wv, wr = S.sn_get_state(whole)
    assert np.array_equal(raster, want), f"first differing step {np.nonzero((raster != want).any(1))[0][:1]}"
    assert np.array_equal(v.view(np.uint32), np.asarray(wv).view(np.uint32)) and np.array_equal(r, wr)
    _, wsp, wev = S.sn_get_counters(whole)
    assert spikes == wsp and events == wev and want[-1].sum() > 0


def test_shard_exchange_rules():
    from paper_2305_02510_gb300 import sn as S
    wl = W.random_small(22, n=100, integer=True, steps=20, max_delay=4, p=0.1)
    wl["delay"] = np.maximum(np.asarray(wl["delay"], np.int32), 2)
    c = S.from_workload_shard(wl, 32, 68, record_steps=20)
    assert S.sn_shard_info(c) == (32, 68, 2)
    with pytest.raises(S.SnError) as e:            # more than the smallest delay at once
        S.sn_run(c, 3)
    assert e.value.status == S.SN_EINVAL
    S.sn_run(c, 2)
    with pytest.raises(S.SnError) as e:            # the other shard's rows are not in yet
        S.sn_run(c, 1)
    assert e.value.status == S.SN_ESTATE
    with pytest.raises(S.SnError) as e:            # rows of steps not run
        S.sn_shard_put_spikes(c, 0, 3, np.zeros((3, 4), np.uint32))
    assert e.value.status == S.SN_EINVAL
    S.sn_shard_put_spikes(c, 0, 2, np.zeros((2, 4), np.uint32))
    S.sn_run(c, 2)
    for bad in (dict(first=16, count=32), dict(first=0, count=40)):
        with pytest.raises(S.SnError) as e:
            S.from_workload_shard(wl, bad["first"], bad["count"])
        assert e.value.status == S.SN_EINVAL
    with pytest.raises(S.SnError) as e:
        S.sn_set_propagation(c, S.SN_PUSH)
    assert e.value.status == S.SN_EUNSUPPORTED
