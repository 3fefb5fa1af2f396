"""Pins for the BPTT reference (oracle/bptt_ref.py):

  * its forward pass equals the C oracle simulator on the same layered
    network (input spikes injected as events into relay neurons), spike for
    spike, for several delay patterns and a refractory period;
  * with a smooth spike (sigmoid) and an attached reset, its autograd
    gradient equals central finite differences of its own forward pass, which
    checks the unrolled delay paths, the leak derivative and the custom
    spike function's backward;
  * torch.autograd.gradcheck of the smooth spike function.
"""

import numpy as np
import pytest
import torch

from oracle import bptt_ref as R, oracle as O
from paper_2305_02510_gb300 import workloads as W


def small_task(seed=0, sizes=(20, 16, 12, 5), B=3, T=40, refractory=0):
    t = W.bptt_task(batch=B, sizes=sizes, steps=T, seed=seed)
    t["refractory"] = refractory
    # stronger input so that every layer spikes
    t["w"] = [w * 1.5 for w in t["w"]]
    return t


def as_simulator_network(task, b):
    """The layered network as one synapse list: layer-0 relay neurons fire
    exactly at the input spikes (event of 1 against threshold 0.5, leak 10)."""
    sizes = task["sizes"]
    off = np.cumsum((0,) + tuple(sizes))
    n = int(off[-1])
    th = np.concatenate([np.full(sizes[0], 0.5)] + [np.full(s, task["threshold"]) for s in sizes[1:]])
    lk = np.concatenate([np.full(sizes[0], 10.0)] + [np.full(s, task["leak"]) for s in sizes[1:]])
    R_ = np.concatenate([np.zeros(sizes[0], np.int32)] + [np.full(s, task["refractory"], np.int32) for s in sizes[1:]])
    wl = W._base(n, "f32", th, lk, task["reset"], R_, task["max_delay"], task["steps"])
    pre, post, w, d = [], [], [], []
    for l, (wm, dm) in enumerate(zip(task["w"], task["delay"])):
        i, j = np.nonzero(np.ones_like(dm, dtype=bool))
        pre.append(i + off[l]); post.append(j + off[l + 1])
        w.append(wm[i, j].astype(np.float64)); d.append(dm[i, j].astype(np.int32))
    wl.update(pre=np.concatenate(pre).astype(np.int32), post=np.concatenate(post).astype(np.int32),
              weight=np.concatenate(w), delay=np.concatenate(d))
    tt, ii = np.nonzero(task["input"][:, b, :])
    wl["events"] = dict(step=tt.astype(np.int32), neuron=ii.astype(np.int32), value=np.ones(tt.size))
    return wl, off


@pytest.mark.parametrize("seed,refractory", [(0, 0), (1, 0), (2, 2)])
def test_forward_equals_simulator_oracle(seed, refractory):
    task = small_task(seed, refractory=refractory)
    ws = [torch.tensor(w, dtype=torch.float64) for w in task["w"]]
    counts, spikes, _ = R.forward(task, ws, record=True)
    total = 0
    for b in range(task["batch"]):
        wl, off = as_simulator_network(task, b)
        _, raster, _ = O.run(wl, O.F64, task["steps"])
        assert np.array_equal(raster[:, :task["sizes"][0]].T, task["input"][:, b, :].T)
        for l in range(1, len(task["sizes"])):
            ref = np.stack([spikes[l][t][b].numpy() for t in range(task["steps"])]).astype(np.uint8)
            assert np.array_equal(raster[:, off[l]:off[l + 1]], ref), (b, l)
            total += int(ref.sum())
        assert np.array_equal(counts[b].numpy(), raster[:, off[-2]:off[-1]].sum(0))
    assert total > 50


def test_smooth_adjoint_matches_finite_differences():
    task = small_task(3, sizes=(10, 9, 7, 4), B=2, T=25)
    loss0, _, grads = R.gradients(task, smooth=5.0, detach_reset=False)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for l, w in enumerate(task["w"]):
        for _ in range(6):
            i, j = rng.integers(0, w.shape[0]), rng.integers(0, w.shape[1])

            def loss_at(delta):
                ws = [torch.tensor(x, dtype=torch.float64) for x in task["w"]]
                ws[l][i, j] += delta
                c = R.forward(task, ws, smooth=5.0, detach_reset=False)
                return float(R.loss_fn(c, task["labels"]))
            fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
            g = float(grads[l][i, j])
            assert abs(fd - g) <= 1e-6 + 1e-5 * abs(g), (l, i, j, fd, g)


def test_smooth_spike_gradcheck():
    x = torch.randn(30, dtype=torch.float64, requires_grad=True)
    m = torch.ones(30, dtype=torch.float64)
    assert torch.autograd.gradcheck(lambda v: R.SurrogateSpike.apply(v, m, 10.0, 5.0, None), (x,))


def test_leak_derivative_rule():
    v = torch.tensor([0.3, 0.04, -0.02, -0.2, 0.0], dtype=torch.float64, requires_grad=True)
    out = R.leak_toward_reset(v, 0.05, 0.0)
    assert torch.allclose(out.detach(), torch.tensor([0.25, 0.0, 0.0, -0.15, 0.0], dtype=torch.float64))
    out.sum().backward()
    assert v.grad.tolist() == [1.0, 0.0, 0.0, 1.0, 0.0]


def test_float32_itself_exceeds_the_state_bound_at_full_size():
    """The reading behind the full-size BPTT state tolerance: over the 100
    integrated steps of the 700-1024-1024-20, batch-128 network, a plain
    float32 evaluation of the reference (same spikes as float64) already
    deviates from float64 by more than 1e-5 * max(|V|, theta) in the first
    hidden layer (about 1.09 of it), so no float32 evaluation can be held to
    the bound itself; the kernels are held to a multiple of this level."""
    task = W.bptt_task()
    T, k = task["steps"], task["checkpoint_every"]
    ws = [torch.tensor(w, dtype=torch.float64) for w in task["w"]]
    _, sp, pre = R.forward(task, ws, record=True)
    given = [[sp[l + 1][t].float() for t in range(T)] for l in range(len(ws))]
    w32 = [torch.tensor(w, dtype=torch.float32) for w in task["w"]]
    _, _, pre32 = R.forward(task, w32, dtype=torch.float32, given=given, record=True)
    th = task["threshold"]
    u = torch.stack([pre[0][t] for t in range(T)]).numpy()
    s = torch.stack([sp[1][t] for t in range(T)]).numpy().astype(bool)
    v = np.where(s, task["reset"], u)[k - 1::k]
    v32 = np.where(s, task["reset"], torch.stack([pre32[0][t] for t in range(T)]).double().numpy())[k - 1::k]
    ratio = np.abs(v32 - v) / (1e-5 * np.maximum(np.abs(v), th))
    assert ratio.max() > 1.0, ratio.max()
    # almost all states are well inside it: the excess is float32 rounding at
    # the largest sums, not a wrong term
    assert np.quantile(ratio, 0.999) < 0.5
