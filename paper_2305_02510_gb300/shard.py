"""Partition of the independent work of one simulation over several GPUs.

Three workloads split without any exchange of simulation data:
  - batched networks: each rank simulates a contiguous range of the networks,
    balanced by work, in one batched context whose Poisson streams are keyed
    by the networks' global indices (sn_set_poisson_stream), so every network
    sees the input it gets in a single context holding them all;
  - one shared dense network driven by many input trains: each rank holds the
    weights and a contiguous range of the trains (a multiple of the tensor-core
    tile, 128), keyed the same way;
  - BPTT training: data parallel over the batch; every rank computes dLoss/dW
    of its samples with the loss scaled by its share of the global batch, and
    one all-reduce (sum) of dW gives the gradient of the global batch.
The only collective is the BPTT all-reduce.  A rank's range depends only on
(count, rank, world), so every rank computes the same partition without
communicating.
"""

from __future__ import annotations

import numpy as np


def contiguous_split(work, world: int) -> np.ndarray:
    """Boundaries b[0] = 0 <= ... <= b[world] = len(work) of `world` contiguous
    ranges with about equal total work: range r ends at the first item whose
    cumulative work reaches (r + 1) / world of the total.  Every item lies in
    exactly one range."""
    w = np.asarray(work, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if w.size and (w < 0).any():
        raise ValueError("work must be non-negative")
    c = np.cumsum(w)
    total = c[-1] if c.size else 0.0
    b = np.zeros(world + 1, np.int64)
    for r in range(1, world):
        b[r] = int(np.searchsorted(c, total * r / world, side="left")) + 1 if total > 0 else (w.size * r) // world
        b[r] = min(max(b[r], b[r - 1]), w.size)
    b[world] = w.size
    return b


def network_work(nets) -> np.ndarray:
    """Work of one batched network per timestep, in memory traffic: its
    neurons' state and its synapses (the update touches every neuron, a spike
    every outgoing synapse)."""
    return np.asarray([w["n"] * 56 + 6 * len(w["pre"]) for w in nets], np.float64)


def network_shard(nets, rank: int, world: int):
    """(first global index, networks) of rank's contiguous range of `nets`."""
    b = contiguous_split(network_work(nets), world)
    return int(b[rank]), nets[b[rank]:b[rank + 1]]


def train_shard(trains: int, rank: int, world: int, align: int = 128):
    """(first train, train count) of rank's range: `trains` split into whole
    blocks of `align` trains, as evenly as the blocks allow (ranks beyond the
    block count get none)."""
    if trains % align:
        raise ValueError(f"trains ({trains}) must be a multiple of {align}")
    blocks = trains // align
    b0 = (blocks * rank) // world
    b1 = (blocks * (rank + 1)) // world
    return b0 * align, (b1 - b0) * align


def batch_shard(batch: int, rank: int, world: int, align: int = 1):
    """(first sample, sample count) of rank's share of a training batch, in
    whole blocks of `align` samples (8 keeps the tensor-core engine)."""
    if batch % align:
        raise ValueError(f"batch ({batch}) must be a multiple of {align}")
    blocks = batch // align
    b0 = (blocks * rank) // world
    b1 = (blocks * (rank + 1)) // world
    return b0 * align, (b1 - b0) * align


def task_slice(task, first: int, count: int):
    """The BPTT task restricted to samples [first, first + count): inputs and
    labels sliced, weights and delays shared."""
    t = dict(task)
    t["input"] = task["input"][:, first:first + count]
    t["labels"] = task["labels"][first:first + count]
    t["batch"] = count
    return t


def data_parallel_backward(loss_of_shard, weights, shard_count: int, batch_total: int, group=None,
                           world: int = 1):
    """Backward of one rank's share of a data-parallel training step.
    loss_of_shard: the mean loss over this rank's samples; it is scaled by
    shard_count / batch_total, so that the gradients summed over the ranks are
    those of the mean loss over the whole batch.  With world > 1 the weights'
    gradients are then all-reduced (sum) over the ranks."""
    (loss_of_shard * (shard_count / batch_total)).backward()
    grads = [w.grad for w in weights]
    if world > 1:
        allreduce_gradients(grads, group)
    return grads


def allreduce_gradients(grads, group=None):
    """Sum each gradient tensor over the ranks in place (one all-reduce per
    tensor)."""
    import torch.distributed as dist
    for g in grads:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return grads


# ---------------------------------------------------------------------------
# One network over several GPUs: each rank simulates a contiguous range of
# the neurons (sn_create_shard) and the ranks exchange spike rows.  A spike of
# step t reaches no neuron before t + d_min (the smallest synaptic delay), so
# a rank advances d_min steps on the rows it has, then every rank's new rows
# are combined (each rank contributes the words of its own neurons) and put
# into every shard before the next d_min steps.

def neuron_shard(n: int, rank: int, world: int):
    """(first, count) of rank's neurons: a contiguous range of whole 32-neuron
    raster words, the words split as evenly as possible (count 0 for ranks
    beyond the word count)."""
    words = (n + 31) // 32
    w0 = words * rank // world
    w1 = words * (rank + 1) // world
    first = w0 * 32
    return first, max(0, min(n, w1 * 32) - first)


def exchange_loop(steps: int, per_exchange: int, run, own_rows, combine, put):
    """Advance `steps` steps in runs of at most `per_exchange` steps; after each
    run of steps [t, t + k): own_rows(t, t + k) gives this rank's rows (its own
    words set, every other word zero), combine(rows) sums them over the ranks
    (the ranks' words are disjoint, so the sum is the whole-network rows), and
    put(t, t + k, rows) installs them.  Returns the steps advanced."""
    t = 0
    while t < steps:
        k = min(per_exchange, steps - t)
        run(k)
        rows = own_rows(t, t + k)
        put(t, t + k, combine(rows))
        t += k
    return t


def run_shard(ctx, steps: int, t_start: int = 0, group=None):
    """Advance the shard context `ctx` (sn_create_shard) by `steps` steps from
    step t_start, exchanging spike rows with the other ranks of `group`
    (torch.distributed; one all-reduce of the new rows per exchange).  Every
    rank calls it with the same steps."""
    import torch
    import torch.distributed as dist
    from . import sn as S
    first, count, k = S.sn_shard_info(ctx)
    w0, w1 = first // 32, (first + count + 31) // 32
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")

    def own_rows(t0, t1):
        full = S.sn_get_spikes(ctx, t_start + t0, t_start + t1)
        rows = np.zeros_like(full)
        rows[:, w0:w1] = full[:, w0:w1]
        return rows

    def combine(rows):
        x = torch.from_numpy(rows.view(np.int32).copy()).to(dev)
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
        return x.cpu().numpy().view(np.uint32)

    return exchange_loop(steps, k, lambda n_: S.sn_run(ctx, n_), own_rows, combine,
                         lambda t0, t1, rows: S.sn_shard_put_spikes(ctx, t_start + t0, t_start + t1, rows))
