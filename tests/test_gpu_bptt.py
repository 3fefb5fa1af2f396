"""BPTT kernels (sn_create_ff / sn_ff_forward / sn_backward behind
SNNFunction) against the float64 unrolled reference trained by torch
autograd (oracle/bptt_ref.py).

Forward: spikes and counts equal the reference's; membrane checkpoints within
1e-5 of max(|V|, theta), or at the full size (100 integrated steps) within
twice the deviation of a plain float32 evaluation of the reference.  Backward: per layer, the Frobenius-relative and the
largest elementwise deviation of dLoss/dW from the float64 reference must be
within max(1e-4, 2 x the deviation of a plain float32 evaluation of the same
reference with the same spike decisions).  (At the full size the first
layer's gradient is ill-conditioned in float32 itself: plain float32 torch
arithmetic deviates from float64 by about 1e-4 there.)  At the full
700-1024-1024-20, batch 128, 100-step size the reference takes the kernels'
spike decisions (teacher forcing); every decision is checked against the
reference's own state first."""

import numpy as np
import pytest

from oracle import bptt_ref as R
from paper_2305_02510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def run_gpu(task, engine=None, recompute=False):
    from paper_2305_02510_gb300 import bptt, sn as S
    net = bptt.FFNet.from_task(task, engine=engine, recompute=recompute)
    dev = torch.device("cuda")
    x = torch.tensor(task["input"], device=dev)
    ws = [torch.tensor(w, device=dev, requires_grad=True) for w in task["w"]]
    counts = bptt.SNNFunction.apply(net, x, *ws)
    loss = torch.nn.functional.cross_entropy(counts, torch.tensor(task["labels"], device=dev))
    loss.backward()
    spikes = [S.sn_ff_get_spikes(net.ctx, l) for l in range(len(task["sizes"]))]
    ck = [None] + [S.sn_ff_get_checkpoints(net.ctx, l) for l in range(1, len(task["sizes"]))]
    return (loss.item(), counts.detach().cpu().numpy(), [w.grad.cpu().numpy() for w in ws], spikes, ck)


def fp32_level(task, given):
    """Deviation of a plain float32 evaluation of the reference (same spike
    decisions) from float64, per layer: (Frobenius-relative, max-abs/scale)."""
    ws64 = [torch.tensor(w, dtype=torch.float64, requires_grad=True) for w in task["w"]]
    ws32 = [torch.tensor(w, dtype=torch.float32, requires_grad=True) for w in task["w"]]
    c64 = R.forward(task, ws64, given=given)
    c32 = R.forward(task, ws32, dtype=torch.float32,
                    given=None if given is None else [[g.float() for g in x] for x in given])
    g64 = torch.autograd.grad(R.loss_fn(c64, task["labels"]), ws64)
    g32 = torch.autograd.grad(R.loss_fn(c32, task["labels"]), ws32)
    out = []
    for a, b in zip(g32, g64):
        a, b = a.double().numpy(), b.numpy()
        out.append((np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()))
    return out


def near_leak_boundary(task, pre, spikes, band=1e-5):
    """Per layer, the neurons whose reference state after some step lies
    within `band` of |V - reset| = leak, where the clamped leak's derivative
    steps from 1 to 0 and float32 and float64 states may fall on different
    sides."""
    out = []
    for l in range(len(pre)):
        u = torch.stack([x.detach() for x in pre[l]]).numpy()
        s = np.asarray(spikes[l + 1], bool)
        V = np.where(s, task["reset"], u)
        gap = np.abs(np.abs(V - task["reset"]) - task["leak"])
        out.append(set(np.nonzero((gap < band).any(axis=(0, 1)))[0].tolist()))
    return out


def compare_grads(g_gpu, g_ref, level, near):
    """Per layer: the Frobenius-relative deviation and the largest elementwise
    deviation (relative to the layer's largest entry) within
    max(1e-4, 2 x plain float32's deviation).  A neuron whose state touches
    the clamped leak's kink (derivative 1 -> 0 at |V - reset| = leak) may
    switch a whole gradient path between float32 and float64, so the
    elementwise check skips those neurons' columns, and applies to a layer
    only when no layer downstream has such neurons; the Frobenius check
    always applies."""
    L = len(g_gpu)
    for l, (a, b) in enumerate(zip(g_gpu, g_ref)):
        b = b.numpy()
        scale = np.abs(b).max()
        assert scale > 0, l
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= max(1e-4, 2 * level[l][0]), (l, rel, level[l])
        if any(near[k] for k in range(l + 1, L)):
            continue
        keep = np.ones(b.shape[1], bool)
        keep[list(near[l])] = False
        dev = np.abs(a - b)[:, keep] / scale
        assert dev.max(initial=0.0) <= max(1e-4, 2 * level[l][1]), (l, float(dev.max()), level[l], len(near[l]))


@pytest.mark.parametrize("seed,k,sizes,B,T", [
    (0, 10, (40, 48, 36, 6), 4, 30),
    (1, 5, (33, 70, 20, 7), 3, 27),
    (2, 10, (64, 32, 32, 10), 5, 40),
    (3, 20, (50, 40, 5), 2, 45),
])
def test_bptt_small_free_running(seed, k, sizes, B, T):
    check_small_free_running(seed, k, sizes, B, T, None)


@pytest.mark.parametrize("seed,k,sizes,B,T", [
    (4, 10, (40, 48, 36, 6), 8, 30),
    (5, 5, (130, 200, 20, 7), 16, 25),
    (6, 20, (64, 129, 10), 8, 40),
])
def test_bptt_small_free_running_tensor(seed, k, sizes, B, T):
    """The tensor-core engine (batches that are multiples of 8), ragged sizes
    across 64-column and 128-row tile edges."""
    check_small_free_running(seed, k, sizes, B, T, "tensor")


def check_small_free_running(seed, k, sizes, B, T, engine):
    task = W.bptt_task(batch=B, sizes=sizes, steps=T, seed=seed)
    task["w"] = [w * 1.5 for w in task["w"]]
    task["checkpoint_every"] = k
    loss, counts, grads, spikes, ck = run_gpu(task, engine)
    ref_loss, ref_counts, ref_grads = R.gradients(task)
    ws = [torch.tensor(w, dtype=torch.float64) for w in task["w"]]
    _, ref_spikes, ref_pre = R.forward(task, ws, record=True)
    near = near_leak_boundary(task, ref_pre, spikes)
    th = task["threshold"]
    for l in range(1, len(sizes)):
        ref = np.stack([ref_spikes[l][t].numpy() for t in range(T)]).astype(np.uint8)
        assert np.array_equal(spikes[l], ref), l
        # membrane checkpoints (state after steps k-1, 2k-1, ...) within
        # 1e-5 * max(|V|, theta) of the float64 reference
        u = torch.stack([ref_pre[l - 1][t].detach() for t in range(T)]).numpy()
        v = np.where(ref.astype(bool), task["reset"], u)[k - 1::k][:ck[l].shape[0]]
        assert ck[l].shape[0] == T // k
        tol = 1e-5 * np.maximum(np.abs(v), th)
        assert np.all(np.abs(ck[l] - v) <= tol), (l, float((np.abs(ck[l] - v) / tol).max()))
    assert spikes[-1].sum() > 0
    assert np.array_equal(counts, ref_counts.numpy())
    assert abs(loss - float(ref_loss)) < 1e-5
    compare_grads(grads, ref_grads, fp32_level(task, None), near)


@pytest.mark.parametrize("engine", ["simt", "tensor"])
def test_bptt_kept_input_equals_recomputed(engine):
    """The backward on the synaptic input kept from the forward and on the
    input recomputed by the forward's own kernel: identical losses, counts,
    spikes, checkpoints and gradients, bit for bit."""
    task = W.bptt_task(batch=16, sizes=(130, 200, 20, 7), steps=25, seed=8)
    task["w"] = [w * 1.5 for w in task["w"]]
    task["checkpoint_every"] = 5
    kept = run_gpu(task, engine)
    again = run_gpu(task, engine, recompute=True)
    assert kept[0] == again[0] and np.array_equal(kept[1], again[1])
    for a, b in zip(kept[2], again[2]):
        assert np.array_equal(a, b)
    for a, b in zip(kept[3], again[3]):
        assert np.array_equal(a, b)
    for a, b in zip(kept[4][1:], again[4][1:]):
        assert np.array_equal(a, b)
    assert kept[3][-1].sum() > 0


@pytest.mark.parametrize("engine", ["simt", "tensor"])
def test_bptt_full_size_teacher_forced(engine):
    task = W.bptt_task()           # 700-1024-1024-20, batch 128, 100 steps, k = 10
    loss, counts, grads, spikes, ck = run_gpu(task, engine)
    T, L = task["steps"], len(task["sizes"]) - 1
    given = [[torch.tensor(spikes[l + 1][t], dtype=torch.float64) for t in range(T)] for l in range(L)]
    ws = [torch.tensor(w, dtype=torch.float64, requires_grad=True) for w in task["w"]]
    ref_counts, _, ref_pre = R.forward(task, ws, given=given, record=True)
    # the same teacher-forced forward in plain float32 arithmetic: over 100
    # integrated steps float32 itself drifts from float64 by about the state
    # tolerance, so the kernels' states are held to max(1e-5 relative, twice
    # plain float32's deviation), as the gradients are
    w32 = [torch.tensor(w, dtype=torch.float32) for w in task["w"]]
    _, _, pre32 = R.forward(task, w32, dtype=torch.float32, given=[[g.float() for g in x] for x in given],
                            record=True)
    # every spike decision of the kernels agrees with the reference's state
    # unless that state lies within 1e-4 * theta of the threshold
    th = task["threshold"]
    flips = 0
    for l in range(L):
        u = torch.stack([ref_pre[l][t].detach() for t in range(T)]).numpy()
        s = spikes[l + 1].astype(bool)
        bad = (u > th) != s
        flips += int(bad.sum())
        assert np.all(np.abs(u[bad] - th) < 1e-4 * th), l
        # checkpoints: state after steps k-1, 2k-1, ...
        k = task["checkpoint_every"]
        v = np.where(s, task["reset"], u)[k - 1::k][:ck[l + 1].shape[0]]
        u32 = torch.stack([pre32[l][t].detach() for t in range(T)]).double().numpy()
        v32 = np.where(s, task["reset"], u32)[k - 1::k][:ck[l + 1].shape[0]]
        tol = 1e-5 * np.maximum(np.abs(v), th) + 1e-6
        level = float((np.abs(v32 - v) / tol).max())
        worst = float((np.abs(ck[l + 1] - v) / tol).max())
        assert worst <= max(1.0, 2.0 * level), (l, worst, level)
        if engine == "simt":
            # the SIMT engine (the simulator's own FP32 order) against the
            # plain bound 1e-5 * max(|V|, theta), no absolute term: within
            # 1.25x of what plain float32 arithmetic reaches (layer 1 of this
            # network: about 1.09 of the bound; tests/test_bptt_ref_pins.py pins
            # that float32 itself exceeds it here)
            plain = 1e-5 * np.maximum(np.abs(v), th)
            lvl = float((np.abs(v32 - v) / plain).max())
            got = float((np.abs(ck[l + 1] - v) / plain).max())
            assert got <= max(1.0, 1.25 * lvl), (l, got, lvl)
    assert spikes[L].sum() > 0
    assert np.array_equal(counts, ref_counts.detach().numpy())
    ref_loss = R.loss_fn(ref_counts, task["labels"])
    ref_grads = torch.autograd.grad(ref_loss, ws)
    near = near_leak_boundary(task, ref_pre, spikes)
    compare_grads(grads, [g.detach() for g in ref_grads], fp32_level(task, given), near)
