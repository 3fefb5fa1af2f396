"""Seeded synthetic workloads for the spiking-network simulator.

This module only draws random networks and input specifications; it holds none
of the simulation arithmetic.  The CUDA library and the CPU oracle both consume
its output, so a test can hand the very same arrays to each side.

The networks stand in for the random Erdos-Renyi graphs the paper benchmarks on
(Section 3): directed Bernoulli(p) connectivity over ordered pairs i != j, or a
fixed out-degree, with the parameter values of each named configuration.

A workload is a plain dict:

    n            number of neurons
    dtype        "f32" (float potentials) or "i32" (exact integer mode)
    threshold, leak, reset : float64 [n]    (integral values in "i32" mode)
    refractory   int32 [n]
    pre, post    int32 [m]   synapse i -> j        (sparse form)
    weight       float64 [m]
    delay        int32 [m]   1 .. max_delay
    dense_w      float32 [n, n] row = pre, column = post (dense form; W_ii = 0)
    dense_delay  int     scalar delay of every dense synapse
    max_delay    int
    poisson      dict(neuron int32[k], rate float64[k], amplitude float64[k], seed int)
    events       dict(step int32[e], neuron int32[e], value float64[e])
    steps        int     number of timesteps the configuration runs
    stdp         None or dict(decay, a_plus, a_minus, wmin, wmax)

Only one of (pre/post/weight/delay) and (dense_w/dense_delay) is present.
"""

from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0x5EED


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def _full(n, v, dt=np.float64):
    return np.full(n, v, dtype=dt)


def bernoulli_pairs(rng, n: int, p: float):
    """Directed pairs (i, j), i != j, each present with probability p.

    Returned sorted by (pre, post).  Rows are drawn in chunks so that large n
    does not materialise an n x n matrix of draws at once.
    """
    pres, posts = [], []
    chunk = max(1, (1 << 22) // max(n, 1))
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        mask = rng.random((r1 - r0, n)) < p
        rows = np.arange(r0, r1)
        mask[rows - r0, rows] = False
        i, j = np.nonzero(mask)
        pres.append((i + r0).astype(np.int32))
        posts.append(j.astype(np.int32))
    if not pres:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.concatenate(pres), np.concatenate(posts)


def fixed_outdegree(rng, n: int, k: int):
    """Exactly k distinct targets per neuron, never itself; sorted by (pre, post)."""
    assert k <= n - 1
    post = np.empty((n, k), dtype=np.int64)
    todo = np.arange(n)
    while todo.size:
        draw = rng.integers(0, n - 1, size=(todo.size, k))
        draw += draw >= todo[:, None]          # skip the diagonal
        draw.sort(axis=1)
        bad = (draw[:, 1:] == draw[:, :-1]).any(axis=1)
        good = ~bad
        post[todo[good]] = draw[good]
        todo = todo[bad]
    pre = np.repeat(np.arange(n, dtype=np.int32), k)
    return pre, post.reshape(-1).astype(np.int32)


def _base(n, dtype, threshold, leak, reset, refractory, max_delay, steps):
    return dict(
        n=int(n), dtype=dtype,
        threshold=np.asarray(threshold, np.float64) * np.ones(n),
        leak=np.asarray(leak, np.float64) * np.ones(n),
        reset=np.asarray(reset, np.float64) * np.ones(n),
        refractory=(np.asarray(refractory) * np.ones(n)).astype(np.int32),
        max_delay=int(max_delay), steps=int(steps), stdp=None,
        events=dict(step=np.zeros(0, np.int32), neuron=np.zeros(0, np.int32),
                    value=np.zeros(0, np.float64)),
        poisson=dict(neuron=np.zeros(0, np.int32), rate=np.zeros(0),
                     amplitude=np.zeros(0), seed=0),
    )


def _poisson(neurons, rate, amplitude, seed):
    neurons = np.asarray(neurons, np.int32)
    k = neurons.size
    return dict(neuron=neurons, rate=np.full(k, float(rate)),
                amplitude=np.full(k, float(amplitude)), seed=int(seed))


# --------------------------------------------------------------------------
# Named configurations
# --------------------------------------------------------------------------

def tiny(integer: bool = False, seed: int = SEED_BASE + 1, steps: int = 1000):
    """Tiny homogeneous net: N=100, p=0.05, delays U{1..4}, theta 1, leak 0.1,
    reset 0, refractory 2; neurons 0..9 Poisson 0.1/step.  The integer copy uses
    weights U{1..5}, theta 10, leak 1 and input amplitude 11."""
    rng = _rng(seed)
    n = 100
    pre, post = bernoulli_pairs(rng, n, 0.05)
    m = pre.size
    delay = rng.integers(1, 5, size=m).astype(np.int32)
    if integer:
        w = rng.integers(1, 6, size=m).astype(np.float64)
        wl = _base(n, "i32", 10, 1, 0, 2, 4, steps)
        amp = 11.0
    else:
        w = rng.random(m)
        wl = _base(n, "f32", 1.0, 0.1, 0.0, 2, 4, steps)
        amp = 2.0
    wl.update(pre=pre, post=post, weight=w, delay=delay)
    wl["poisson"] = _poisson(np.arange(10), 0.1, amp, seed * 7 + 1)
    wl["name"] = "tiny-int" if integer else "tiny"
    return wl


def large_sparse(integer: bool = False, n: int = 100_000, k: int = 100,
                 seed: int = SEED_BASE + 2, steps: int = 1000, n_input: int | None = None):
    """Large sparse net: N=100,000, exactly 100 distinct targets per neuron,
    weights N(0.5, 0.1) clipped to >= 1e-3 with 20% negated, delays U{1..16},
    thresholds U(0.8, 1.2), leak 0.1, refractory 2; Poisson 0.05/step into 1% of
    the neurons with amplitude 2.  Integer variant: weights U{-3..5},
    threshold 20, leak 1, amplitude 21."""
    rng = _rng(seed)
    pre, post = fixed_outdegree(rng, n, k)
    m = pre.size
    delay = rng.integers(1, 17, size=m).astype(np.int32)
    if integer:
        w = rng.integers(-3, 6, size=m).astype(np.float64)
        wl = _base(n, "i32", 20, 1, 0, 2, 16, steps)
        amp = 21.0
    else:
        w = np.maximum(rng.normal(0.5, 0.1, size=m), 1e-3)
        w[rng.random(m) < 0.2] *= -1.0
        th = rng.uniform(0.8, 1.2, size=n)
        wl = _base(n, "f32", th, 0.1, 0.0, 2, 16, steps)
        amp = 2.0
    wl.update(pre=pre, post=post, weight=w, delay=delay)
    ni = n_input if n_input is not None else max(1, n // 100)
    inputs = np.sort(rng.choice(n, size=ni, replace=False)).astype(np.int32)
    wl["poisson"] = _poisson(inputs, 0.05, amp, seed * 7 + 2)
    wl["name"] = "large-sparse-int" if integer else "large-sparse"
    return wl


def large_dense(n: int = 16384, stdp: bool = False, seed: int = SEED_BASE + 3,
                steps: int = 1000):
    """Large dense net: all-to-all N(0, 0.02) weights (W_ii = 0), delay 1,
    theta 1, leak 0.05, refractory 1; Poisson 0.02/step on every neuron with
    amplitude 2.  With stdp=True: pair-based STDP with trace decay 0.9,
    A+ = 0.01, A- = 0.012, weights clipped to [-1, 1]."""
    rng = _rng(seed)
    w = np.empty((n, n), dtype=np.float32)
    rows = max(1, (1 << 24) // n)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        w[r0:r1] = rng.normal(0.0, 0.02, size=(r1 - r0, n)).astype(np.float32)
    np.fill_diagonal(w, 0.0)
    wl = _base(n, "f32", 1.0, 0.05, 0.0, 1, 1, steps)
    wl.update(dense_w=w, dense_delay=1)
    wl["poisson"] = _poisson(np.arange(n), 0.02, 2.0, seed * 7 + 3)
    if stdp:
        wl["stdp"] = dict(decay=0.9, a_plus=0.01, a_minus=0.012, wmin=-1.0, wmax=1.0)
    wl["name"] = "large-dense-stdp" if stdp else "large-dense"
    return wl


def huge_dense(n: int = 100_000, seed: int = SEED_BASE + 7, steps: int = 1000):
    """All-to-all network too large to build on the host (the paper runs a
    100,000-neuron all-to-all network, Section 4): weights N(0, sigma^2) with
    sigma = 0.02 * sqrt(16384 / n), which keeps large-dense's per-step input
    variance, W_ii = 0, delay 1, theta 1, leak 0.05, refractory 1; Poisson
    0.02/step into every neuron at amplitude 2.  The weights are drawn on the
    device by dense_weights_on_device (n = 100,000: 40 GB)."""
    wl = _base(n, "f32", 1.0, 0.05, 0.0, 1, 1, steps)
    wl.update(dense_w_device=dict(seed=int(seed), sigma=0.02 * math.sqrt(16384.0 / n)), dense_delay=1)
    wl["poisson"] = _poisson(np.arange(n), 0.02, 2.0, seed * 7 + 3)
    wl["name"] = f"huge-dense-n{n}"
    return wl


def dense_integer_valued(n: int, seed: int = SEED_BASE + 8, steps: int = 1000, on_device: bool = False):
    """All-to-all network whose float32 weights are the integers -1, 0, +1
    (each nonzero with probability 500 / n, W_ii = 0), theta 8, leak 1,
    reset 0, refractory 1, delay 1; Poisson 0.02/step into every neuron at
    amplitude 9.  Every partial sum of a step's synaptic input is an integer
    far below 2^24, so float32 arithmetic is exact in any order of addition
    and a run must equal the oracle bit for bit whatever the kernel's blocking.
    About 15% of the neurons fire per step, most of them through synaptic
    input.  on_device: the weights are drawn on the device by
    dense_weights_on_device (for sizes beyond a host copy)."""
    q = min(0.5, 500.0 / n)
    wl = _base(n, "f32", 8.0, 1.0, 0.0, 1, 1, steps)
    if on_device:
        wl.update(dense_w_device=dict(seed=int(seed), int_q=q), dense_delay=1)
    else:
        rng = _rng(seed)
        w = np.empty((n, n), dtype=np.float32)
        rows = max(1, (1 << 24) // n)
        for r0 in range(0, n, rows):
            r1 = min(n, r0 + rows)
            u = rng.random((r1 - r0, n))
            w[r0:r1] = (u < q).astype(np.float32) - (u >= 1.0 - q).astype(np.float32)
        np.fill_diagonal(w, 0.0)
        wl.update(dense_w=w, dense_delay=1)
    wl["poisson"] = _poisson(np.arange(n), 0.02, 9.0, seed * 7 + 3)
    wl["name"] = f"dense-integer-valued-n{n}"
    return wl


def dense_weights_on_device(wl, torch, device="cuda"):
    """Device tensor [n, n] float32 with the weights of a huge_dense (or an
    on-device dense_integer_valued) workload, drawn by a seeded torch
    generator on the device (W_ii = 0)."""
    spec, n = wl["dense_w_device"], wl["n"]
    g = torch.Generator(device=device)
    g.manual_seed(spec["seed"])
    w = torch.empty((n, n), dtype=torch.float32, device=device)
    if "int_q" in spec:
        # dense_integer_valued: -1, 0, +1 with P(+1) = P(-1) = q, row block by row block
        q = float(spec["int_q"])
        rows = max(1, (1 << 28) // n)
        for r0 in range(0, n, rows):
            blk = w[r0:r0 + rows]
            blk.uniform_(0.0, 1.0, generator=g)
            blk.copy_((blk < q).float() - (blk >= 1.0 - q).float())
    else:
        w.normal_(0.0, spec["sigma"], generator=g)
    w.fill_diagonal_(0.0)
    return w


def paper_grid(n: int, p: float, seed: int = SEED_BASE + 6, steps: int = 1000,
               amplitude: float = 2.0):
    """The paper's benchmark workload (Section 3): Bernoulli(p) digraph, 3 random
    input neurons each spiked externally every 10 steps, threshold 1, reset 0,
    refractory 0, all weights and delays 1.  The leak is unstated; 0 is used."""
    rng = _rng(seed)
    pre, post = bernoulli_pairs(rng, n, p)
    m = pre.size
    wl = _base(n, "f32", 1.0, 0.0, 0.0, 0, 1, steps)
    wl.update(pre=pre, post=post, weight=np.ones(m), delay=np.ones(m, np.int32))
    inputs = np.sort(rng.choice(n, size=3, replace=False)).astype(np.int32)
    st = np.arange(0, steps, 10, dtype=np.int32)
    wl["events"] = dict(step=np.repeat(st, 3), neuron=np.tile(inputs, st.size),
                        value=np.full(3 * st.size, amplitude))
    wl["name"] = f"paper-grid-n{n}-p{p}"
    return wl


def random_small(seed: int, n: int | None = None, integer: bool = True,
                 max_delay: int | None = None, steps: int = 200, p: float | None = None,
                 events_rate: float = 0.1):
    """Small random nets with heterogeneous parameters and explicit input
    events, used for exhaustive parity and formulation-agreement tests."""
    rng = _rng(seed)
    n = int(n if n is not None else rng.integers(2, 21))
    D = int(max_delay if max_delay is not None else rng.integers(1, 5))
    p = float(p if p is not None else rng.uniform(0.1, 0.6))
    pre, post = bernoulli_pairs(rng, n, p)
    m = pre.size
    delay = rng.integers(1, D + 1, size=m).astype(np.int32)
    if integer:
        w = rng.integers(-3, 6, size=m).astype(np.float64)
        th = rng.integers(1, 8, size=n).astype(np.float64)
        lk = rng.integers(0, 3, size=n).astype(np.float64)
        rs = rng.integers(-2, 1, size=n).astype(np.float64)
        amp_hi = 10
        dt = "i32"
    else:
        w = rng.normal(0.3, 0.5, size=m)
        th = rng.uniform(0.5, 1.5, size=n)
        lk = rng.uniform(0.0, 0.2, size=n)
        rs = rng.uniform(-0.2, 0.0, size=n)
        amp_hi = None
        dt = "f32"
    R = rng.integers(0, 4, size=n).astype(np.int32)
    wl = _base(n, dt, th, lk, rs, R, D, steps)
    wl.update(pre=pre, post=post, weight=w, delay=delay)
    ne = rng.binomial(steps * n, min(1.0, events_rate / max(n, 1) * 3))
    st = rng.integers(0, steps, size=ne).astype(np.int32)
    nu = rng.integers(0, n, size=ne).astype(np.int32)
    if integer:
        val = rng.integers(1, amp_hi, size=ne).astype(np.float64)
    else:
        val = rng.uniform(0.5, 2.5, size=ne)
    wl["events"] = dict(step=st, neuron=nu, value=val)
    wl["name"] = f"random-small-{seed}"
    return wl


def bernoulli_pairs_skip(rng, n: int, p: float):
    """Directed pairs (i, j), i != j, each present with probability p, drawn
    by geometric gaps between successive present pairs in row-major order of
    the n(n-1) off-diagonal positions (the same Bernoulli process as
    bernoulli_pairs at O(m) cost).  Sorted by (pre, post)."""
    total = n * (n - 1)
    if total == 0 or p <= 0.0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    mean = total * p
    chunks = []
    last = -1
    while True:
        k = int(mean - (last + 1) * p + 6.0 * math.sqrt(mean + 1.0) + 64)
        gaps = rng.geometric(p, size=max(k, 64))
        pos = last + np.cumsum(gaps, dtype=np.int64)
        done = pos[-1] >= total
        pos = pos[pos < total]
        chunks.append(pos)
        if done:
            break
        last = int(pos[-1]) if pos.size else last
    lin = np.concatenate(chunks)
    i = lin // (n - 1)
    jj = lin - i * (n - 1)
    j = jj + (jj >= i)
    return i.astype(np.int32), j.astype(np.int32)


def batched_nets(count: int = 4096, seed: int = SEED_BASE + 4, steps: int = 500,
                 nmin: int = 64, nmax: int = 4096, first: int = 0):
    """Independent nets for the batched simulation: N log-uniform in
    [nmin, nmax], connection probability U(0.01, 0.2), thresholds U(0.5, 1.5),
    leaks U(0, 0.2), reset 0, refractory U{0..3}, delays U{1..8}, weights
    N(0, 1)/sqrt(p N); Poisson 0.05/step into 10% of each net's neurons with
    amplitude 2 * max threshold.  The sizes and probabilities of networks
    0 .. first + count - 1 come from one stream (so they depend on
    first + count); network b then draws its synapses and parameters from its
    own seed sequence (seed, b).  Weights are float32, indices int32.
    Returns a list of workload dicts for networks first .. first + count - 1."""
    top = np.random.default_rng(np.random.SeedSequence(int(seed)))
    sizes = np.floor(np.exp(top.uniform(math.log(nmin), math.log(nmax), size=first + count)))
    probs = top.uniform(0.01, 0.2, size=first + count)
    nets = []
    for b in range(first, first + count):
        n = int(min(nmax, max(nmin, sizes[b])))
        p = float(probs[b])
        sub = np.random.default_rng(np.random.SeedSequence([int(seed), b]))
        pre, post = bernoulli_pairs_skip(sub, n, p)
        m = pre.size
        delay = sub.integers(1, 9, size=m).astype(np.int32)
        w = (sub.standard_normal(size=m, dtype=np.float32) / np.float32(math.sqrt(p * n)))
        th = sub.uniform(0.5, 1.5, size=n)
        lk = sub.uniform(0.0, 0.2, size=n)
        R = sub.integers(0, 4, size=n).astype(np.int32)
        wl = _base(n, "f32", th, lk, 0.0, R, 8, steps)
        wl.update(pre=pre, post=post, weight=w, delay=delay)
        ni = max(1, n // 10)
        inputs = np.sort(sub.choice(n, size=ni, replace=False)).astype(np.int32)
        wl["poisson"] = _poisson(inputs, 0.05, 2.0 * float(np.float32(th).max()), seed * 7 + 4)
        wl["net_index"] = b
        wl["name"] = f"batched-{b}"
        nets.append(wl)
    return nets


def shared_dense_i8(n: int = 8192, batch: int = 256, seed: int = SEED_BASE + 5,
                    steps: int = 500):
    """One shared dense integer net driven by `batch` independent Poisson input
    trains: int8 weights U{-8..8} (W_ii = 0), threshold 40, leak 1, reset 0,
    refractory 1, delay 1; every neuron of every train receives Poisson
    0.05/step input with amplitude 41.  Train b uses hash stream b."""
    rng = _rng(seed)
    w = rng.integers(-8, 9, size=(n, n), dtype=np.int8)
    np.fill_diagonal(w, 0)
    wl = _base(n, "i32", 40, 1, 0, 1, 1, steps)
    wl.update(dense_w_i8=w, dense_delay=1, batch=int(batch))
    wl["poisson"] = _poisson(np.arange(n), 0.05, 41.0, seed * 7 + 5)
    wl["name"] = "shared-dense-i8"
    return wl


def to_dense(wl):
    """Dense weight matrix [n, n] (float64) of a sparse workload; duplicate
    (pre, post) pairs are summed.  Only meaningful when every delay equals 1."""
    n = wl["n"]
    w = np.zeros((n, n))
    np.add.at(w, (wl["pre"], wl["post"]), wl["weight"])
    return w


def bptt_task(batch: int = 128, sizes=(700, 1024, 1024, 20), steps: int = 100,
              max_delay: int = 4, seed: int = SEED_BASE + 7, classes: int | None = None):
    """Feedforward spiking network trained by backpropagation through time:
    LIF layers sizes[1..] fed by sizes[0] input channels; weights
    Kaiming-normal N(0, 2/fan_in) (float32), per-synapse delays U{1..max_delay};
    threshold 1, leak 0.05, reset 0, refractory 0; fast-sigmoid surrogate with
    slope 10; membrane checkpoints every 10 steps.  Inputs are Poisson spike
    trains with a rate U(0, 0.2) per (sample, channel); labels uniform over the
    output classes.  Returns a dict with input [steps, batch, n0] uint8,
    labels [batch] int64, w (list of float32 [n_in, n_out]) and delay (list of
    uint8 [n_in, n_out])."""
    rng = _rng(seed)
    sizes = tuple(int(x) for x in sizes)
    rates = rng.uniform(0.0, 0.2, size=(batch, sizes[0]))
    x = (rng.random((steps, batch, sizes[0])) < rates[None]).astype(np.uint8)
    ncls = classes if classes is not None else sizes[-1]
    labels = rng.integers(0, ncls, size=batch).astype(np.int64)
    ws, ds = [], []
    for a, b in zip(sizes[:-1], sizes[1:]):
        ws.append((rng.standard_normal((a, b)) * math.sqrt(2.0 / a)).astype(np.float32))
        ds.append(rng.integers(1, max_delay + 1, size=(a, b)).astype(np.uint8))
    return dict(sizes=sizes, batch=int(batch), steps=int(steps), max_delay=int(max_delay),
                input=x, labels=labels, w=ws, delay=ds, threshold=1.0, leak=0.05, reset=0.0,
                refractory=0, slope=10.0, checkpoint_every=10, name="bptt")
