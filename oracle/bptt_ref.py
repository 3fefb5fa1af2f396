"""Plain unrolled reference of the spiking network's forward pass and of its
surrogate-gradient backward pass (backpropagation through time).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the library's BPTT kernels.
It is plain PyTorch on the CPU in float64, one timestep and one layer at a
time, differentiated by torch autograd.

The forward pass is the simulator's timestep (SuperNeuro Section 2.1 order:
constant leak toward the reset state, add the delayed synaptic input, compare
with the threshold strictly, zero the spikes of refractory neurons, reset)
applied layer by layer to a feedforward network whose synapse i -> j of
layer l has weight W_l[i, j] and delay D_l[i, j] >= 1, so a spike of layer
l-1 at step t reaches layer l at step t + D_l[i, j].  Layer 0 is the input
spike train itself.  The output is the spike count of each output neuron.

Training (not in the paper; its motivation only names SNN training): the
spike's derivative is replaced by the fast-sigmoid surrogate
1 / (1 + slope * |u - theta|)^2; the reset is detached (V = u (1 - s) +
reset * s with s held constant there); the refractory mask is constant; the
clamped leak has derivative 1 where |V - reset| > leak and 0 elsewhere; the
integer delays get no gradient.
"""

from __future__ import annotations

import torch


class SurrogateSpike(torch.autograd.Function):
    """s = [x > 0] * mask forward; ds/dx = mask / (1 + slope |x|)^2 backward.
    With `smooth` > 0 the forward is sigmoid(smooth * x) * mask instead and the
    backward its exact derivative (used to check the adjoint against finite
    differences)."""

    @staticmethod
    def forward(ctx, x, mask, slope, smooth, given):
        ctx.save_for_backward(x, mask)
        ctx.slope, ctx.smooth = slope, smooth
        if given is not None:
            return given
        if smooth > 0:
            return torch.sigmoid(smooth * x) * mask
        return (x > 0).to(x.dtype) * mask

    @staticmethod
    def backward(ctx, g):
        x, mask = ctx.saved_tensors
        if ctx.smooth > 0:
            sg = torch.sigmoid(ctx.smooth * x)
            d = ctx.smooth * sg * (1 - sg)
        else:
            d = 1.0 / (1.0 + ctx.slope * x.abs()) ** 2
        return g * mask * d, None, None, None, None


def leak_toward_reset(v, leak, reset):
    """Constant leak toward the reset state, clamped there (Section 2.1):
    V - leak above reset, V + leak below, reset once within `leak` of it.  The
    derivative is 1 where |V - reset| > leak and 0 elsewhere."""
    d = v - reset
    far = d.abs().detach() > leak
    return torch.where(far, v - leak * torch.sign(d.detach()), torch.full_like(v, reset))


def forward(task, ws, *, dtype=torch.float64, smooth=0.0, detach_reset=True, given=None,
            record=False):
    """Unrolled forward.  ws: list of weight tensors [n_in, n_out] (requires
    grad as needed).  given: optional list (per layer) of [T, B, n] spike
    tensors to use as the spike decisions (teacher forcing); the surrogate
    still acts on this reference's own membrane state.  Returns the output
    counts [B, n_out] (and per-layer spikes and pre-reset states if record)."""
    T, B = task["steps"], task["batch"]
    sizes = task["sizes"]
    th, lk, rs, R = float(task["threshold"]), float(task["leak"]), float(task["reset"]), int(task["refractory"])
    D = task["max_delay"]
    x = torch.as_tensor(task["input"], dtype=dtype)
    masks = []
    for l in range(len(ws)):
        dl = torch.as_tensor(task["delay"][l].astype("int64"))
        masks.append([(dl == d).to(dtype) for d in range(1, D + 1)])
    spikes = [[x[t] for t in range(T)]]
    pre = []
    V = [torch.full((B, n), rs, dtype=dtype) for n in sizes[1:]]
    r = [torch.zeros((B, n), dtype=torch.int64) for n in sizes[1:]]
    counts = torch.zeros((B, sizes[-1]), dtype=dtype)
    for l in range(len(ws)):
        spikes.append([None] * T)
        pre.append([None] * T)
    for t in range(T):
        for l in range(len(ws)):
            I = torch.zeros((B, sizes[l + 1]), dtype=dtype)
            for d in range(1, D + 1):
                if t - d >= 0:
                    I = I + spikes[l][t - d] @ (ws[l] * masks[l][d - 1])
            u = leak_toward_reset(V[l], lk, rs) + I
            mask = (r[l] == 0).to(dtype)
            g = None if given is None else torch.as_tensor(given[l][t], dtype=dtype)
            s = SurrogateSpike.apply(u - th, mask, float(task["slope"]), smooth, g)
            sd = s.detach() if detach_reset else s
            V[l] = u * (1 - sd) + rs * sd
            fired = s.detach() > 0.5
            r[l] = torch.where(fired, torch.full_like(r[l], R), torch.clamp(r[l] - 1, min=0))
            spikes[l + 1][t] = s
            pre[l][t] = u
        counts = counts + spikes[-1][t]
    if record:
        return counts, spikes, pre
    return counts


def loss_fn(counts, labels):
    """Cross-entropy of the output spike counts (as logits) against labels,
    averaged over the batch."""
    return torch.nn.functional.cross_entropy(counts, torch.as_tensor(labels))


def gradients(task, *, dtype=torch.float64, smooth=0.0, detach_reset=True, given=None):
    """(loss, counts, [dL/dW_l]) by autograd through the unrolled forward."""
    ws = [torch.tensor(w, dtype=dtype, requires_grad=True) for w in task["w"]]
    counts = forward(task, ws, dtype=dtype, smooth=smooth, detach_reset=detach_reset, given=given)
    loss = loss_fn(counts, task["labels"])
    grads = torch.autograd.grad(loss, ws)
    return loss.detach(), counts.detach(), [g.detach() for g in grads]
