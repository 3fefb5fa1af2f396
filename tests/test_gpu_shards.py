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
