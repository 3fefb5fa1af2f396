"""Two further formulations of the same simulation, for small networks only.

TEST INFRASTRUCTURE ONLY.  They exist to pin the C oracle to something other
than itself: the paper describes two execution modes, and both must yield the
same spike rasters as the oracle's delay-history form.

* `mat_proxy`: the matrix mode (Section 2.1).  Delays are removed by proxy
  neurons: a synapse of delay d becomes a chain of d-1 private proxy neurons
  with threshold 0, an unbounded leak and no refractory period, so every hop
  has delay 1.  The first d-1 hops have weight 1 and the last hop carries w
  (the paper says every hop has unit weight, which would lose w; the last hop
  must carry it).  Each step is then: leak, add s(t-1) @ W, add the external
  input, compare with the thresholds, zero the spikes of refractory neurons.
  Integer mode uses exact int64 arithmetic; float mode uses float64.

* `abm_registers`: the agent mode (Section 2.2) written out literally with one
  shift register per synapse: the neuron step integrates and fires, a spiking
  neuron writes a 1 into the head of each outgoing register, and the synapse
  step shifts the registers and delivers the final element times the weight
  to the post-neuron on the next step.  Pure Python loops.

Both use the same external-input rules as the oracle: explicit events of
(t, j) summed in the order given; no Poisson sources here.
"""

from __future__ import annotations

import numpy as np


def _leak(v, leak, reset):
    """Constant leak toward the reset state, clamped at it (Section 2.1)."""
    out = v.copy()
    gt, lt = v > reset, v < reset
    out[gt] = np.maximum(v[gt] - leak[gt], reset[gt])
    out[lt] = np.minimum(v[lt] + leak[lt], reset[lt])
    out[~(gt | lt)] = reset[~(gt | lt)]
    return out


def _ext_table(wl, steps, n, dt):
    ext = np.zeros((steps, n), dtype=dt)
    ev = wl["events"]
    for t, j, val in zip(ev["step"], ev["neuron"], ev["value"]):
        if 0 <= t < steps:
            ext[t, j] += dt(val) if dt is not object else val
    return ext


def mat_proxy(wl, steps: int, integer: bool = True):
    """Matrix-mode simulation with proxy neurons.  Returns the raster of the
    original neurons, shape [steps, n], and their final state."""
    n = wl["n"]
    dt = np.int64 if integer else np.float64
    pre, post = np.asarray(wl["pre"]), np.asarray(wl["post"])
    w, d = np.asarray(wl["weight"]), np.asarray(wl["delay"])
    # axonal delays (Section 2.2): neuron i's spikes first cross a chain of
    # axonal_delay[i] proxies shared by all of its outgoing synapses
    ax = np.asarray(wl.get("axonal_delay") if wl.get("axonal_delay") is not None else np.zeros(n), np.int64)
    n_proxy = int(np.sum(np.maximum(d - 1, 0))) + int(ax.sum())
    tot = n + n_proxy
    W = np.zeros((tot, tot), dtype=dt)
    nxt = n
    axon_end = np.arange(n)
    for i in range(n):
        src = i
        for _ in range(int(ax[i])):
            W[src, nxt] += 1
            src = nxt
            nxt += 1
        axon_end[i] = src
    for i, j, wk, dk in zip(pre, post, w, d):
        src = int(axon_end[int(i)])
        for _ in range(int(dk) - 1):          # proxy chain, unit-weight hops
            W[src, nxt] += 1
            src = nxt
            nxt += 1
        W[src, int(j)] += dt(wk)              # the last hop carries w
    big = dt(2**40) if integer else np.inf
    th = np.concatenate([np.asarray(wl["threshold"], dt), np.zeros(n_proxy, dt)])
    lk = np.concatenate([np.asarray(wl["leak"], dt), np.full(n_proxy, big, dt)])
    rs = np.concatenate([np.asarray(wl["reset"], dt), np.zeros(n_proxy, dt)])
    R = np.concatenate([np.asarray(wl["refractory"], np.int64), np.zeros(n_proxy, np.int64)])
    ext = np.zeros((steps, tot), dt)
    ext[:, :n] = _ext_table(wl, steps, n, dt)
    V = rs.copy()
    r = np.zeros(tot, np.int64)
    s = np.zeros(tot, dt)
    raster = np.zeros((steps, n), np.uint8)
    for t in range(steps):
        V = _leak(V, lk, rs)
        V = V + s @ W
        V = V + ext[t]
        c = V > th
        fire = c & (r == 0)
        V = np.where(fire, rs, V)
        r = np.where(fire, R, np.maximum(r - 1, 0))
        s = fire.astype(dt)
        raster[t] = fire[:n]
    return raster, V[:n], r[:n]


def abm_registers(wl, steps: int):
    """Agent-mode simulation with explicit per-synapse delay registers, in
    pure Python (exact for integer workloads).  Returns the raster [steps, n]
    and the final state."""
    n = wl["n"]
    pre = [int(x) for x in wl["pre"]]
    post = [int(x) for x in wl["post"]]
    w = [float(x) for x in wl["weight"]]
    d = [int(x) for x in wl["delay"]]
    th = [float(x) for x in wl["threshold"]]
    lk = [float(x) for x in wl["leak"]]
    rs = [float(x) for x in wl["reset"]]
    R = [int(x) for x in wl["refractory"]]
    regs = [[0] * dk for dk in d]              # register k, element 0 = head
    out_syn = [[] for _ in range(n)]
    for k, i in enumerate(pre):
        out_syn[i].append(k)
    ext = [[0.0] * n for _ in range(steps)]
    ev = wl["events"]
    for t, j, val in zip(ev["step"], ev["neuron"], ev["value"]):
        if 0 <= t < steps:
            ext[int(t)][int(j)] += float(val)
    V = list(rs)
    r = [0] * n
    raster = np.zeros((steps, n), np.uint8)
    for t in range(steps):
        # synapse step of the previous step's end: deliver final elements
        syn_in = [0.0] * n
        for k in range(len(pre)):
            if regs[k][-1]:
                syn_in[post[k]] += w[k]
        # neuron step
        fired = [False] * n
        for j in range(n):
            v = V[j]
            if v > rs[j]:
                v = max(v - lk[j], rs[j])
            elif v < rs[j]:
                v = min(v + lk[j], rs[j])
            v = v + syn_in[j]
            v = v + ext[t][j]
            if v > th[j] and r[j] == 0:
                fired[j] = True
                v = rs[j]
                r[j] = R[j]
            elif r[j] > 0:
                r[j] -= 1
            V[j] = v
            raster[t, j] = fired[j]
        # synapse step: shift every register, spiking pre writes the head
        for k in range(len(pre)):
            regs[k] = [1 if fired[pre[k]] else 0] + regs[k][:-1]
    return raster, np.array(V), np.array(r, np.int32)
