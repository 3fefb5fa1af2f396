"""Training of a feedforward spiking network by backpropagation through time
on the library's kernels: the forward pass is the simulator's timestep
(exact spikes), the backward pass is the hand-written surrogate-gradient
adjoint.  torch provides the tensors and the autograd graph only."""

from __future__ import annotations

import torch

from . import sn as S


class FFNet:
    """One sn_create_ff context: layer sizes, per-synapse delays and the
    shared neuron parameters are fixed; the weights are passed per call."""

    def __init__(self, sizes, delays, *, batch, steps, threshold=1.0, leak=0.05, reset=0.0,
                 refractory=0, slope=10.0, checkpoint_every=10, device="cuda", engine=None,
                 recompute=False):
        """engine: None or "auto" (tensor cores where the shapes allow), "simt"
        or "tensor" (sn_ff_set_engine).  recompute: the backward recomputes
        each layer's synaptic input instead of keeping it from the forward."""
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        self.ctx = S.sn_create_ff(sizes, delays, threshold=threshold, leak=leak, reset=reset,
                                  refractory=refractory, slope=slope, checkpoint_every=checkpoint_every,
                                  batch=batch, steps=steps, stream=self.stream.cuda_stream,
                                  recompute=recompute)
        if engine is not None:
            S.sn_ff_set_engine(self.ctx, {"auto": S.SN_FF_AUTO, "simt": S.SN_FF_SIMT,
                                          "tensor": S.SN_FF_TENSOR}[engine])
        self.sizes, self.batch, self.steps = list(sizes), batch, steps

    @classmethod
    def from_task(cls, task, **kw):
        return cls(task["sizes"], task["delay"], batch=task["batch"], steps=task["steps"],
                   threshold=task["threshold"], leak=task["leak"], reset=task["reset"],
                   refractory=task["refractory"], slope=task["slope"],
                   checkpoint_every=task["checkpoint_every"], **kw)

    def forward(self, x, weights):
        counts = torch.empty((self.batch, self.sizes[-1]), dtype=torch.float32, device=self.device)
        S.sn_ff_forward(self.ctx, x, weights, counts)
        return counts

    def backward(self, grad_counts, weights):
        grads = [torch.empty_like(w) for w in weights]
        S.sn_backward(self.ctx, grad_counts.contiguous(), grads)
        return grads


class SNNFunction(torch.autograd.Function):
    """counts = SNNFunction.apply(net, x, W_1, ..., W_L): output spike counts
    [batch, n_L] of the network for input spikes x (CUDA uint8
    [steps, batch, n_0]); the backward returns dLoss/dW_l from the adjoint
    kernels."""

    @staticmethod
    def forward(ctx, net, x, *weights):
        ws = [w.contiguous() for w in weights]
        ctx.net = net
        ctx.save_for_backward(*ws)
        return net.forward(x.contiguous(), ws)

    @staticmethod
    def backward(ctx, grad_counts):
        ws = ctx.saved_tensors
        grads = ctx.net.backward(grad_counts, list(ws))
        return (None, None, *grads)
