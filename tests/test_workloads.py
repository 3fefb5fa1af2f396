"""The seeded input recipes that stand in for the paper's workloads
(Section 3 and the configurations built on it): shapes, value ranges,
distributions and determinism of every generator, at sizes small enough for
the CPU suite.  The generators hold none of the simulation's arithmetic."""

import math

import numpy as np
import pytest

from paper_2305_02510_gb300 import workloads as W


def within(count, mean, var, k=6.0):
    """count lies within k standard deviations of its mean."""
    return abs(count - mean) <= k * math.sqrt(var) + 1.0


def pair_keys(pre, post, n):
    return pre.astype(np.int64) * n + post


@pytest.mark.parametrize("gen", [W.bernoulli_pairs, W.bernoulli_pairs_skip])
@pytest.mark.parametrize("n,p", [(50, 0.1), (300, 0.02), (40, 0.9), (200, 0.5)])
def test_bernoulli_pairs(gen, n, p):
    """Directed pairs without self-loops, sorted and distinct, each present
    with probability p: the edge count within 6 sigma of p n (n - 1), and
    in-degrees spread like Binomial(n - 1, p)."""
    pre, post = gen(W._rng(123 + n), n, p)
    assert pre.dtype == np.int32 and post.dtype == np.int32
    assert np.all(pre != post)
    assert np.all((pre >= 0) & (pre < n) & (post >= 0) & (post < n))
    assert np.all(np.diff(pair_keys(pre, post, n)) > 0)
    tot = n * (n - 1)
    assert within(pre.size, p * tot, tot * p * (1 - p)), (pre.size, p * tot)
    indeg = np.bincount(post, minlength=n)
    var = (n - 1) * p * (1 - p)
    assert 0.5 * var <= indeg.var() <= 1.6 * var, (indeg.var(), var)


def test_bernoulli_pairs_extremes():
    """p = 1 gives every off-diagonal pair exactly once; p = 0 none."""
    for gen in (W.bernoulli_pairs, W.bernoulli_pairs_skip):
        pre, post = gen(W._rng(1), 23, 1.0)
        assert pre.size == 23 * 22
        want = np.array([(i, j) for i in range(23) for j in range(23) if i != j])
        assert np.array_equal(np.stack([pre, post], 1), want)
        pre, post = gen(W._rng(1), 23, 0.0)
        assert pre.size == 0


def test_fixed_outdegree():
    pre, post = W.fixed_outdegree(W._rng(7), 500, 20)
    assert pre.size == 500 * 20
    assert np.array_equal(np.bincount(pre, minlength=500), np.full(500, 20))
    assert np.all(pre != post)
    assert np.all(np.diff(pair_keys(pre, post, 500)) > 0)      # distinct, sorted


@pytest.mark.parametrize("integer", [False, True])
def test_tiny(integer):
    wl = W.tiny(integer=integer)
    n, m = wl["n"], wl["pre"].size
    assert n == 100 and wl["max_delay"] == 4
    assert within(m, 0.05 * 9900, 9900 * 0.05 * 0.95)
    assert set(np.unique(wl["delay"])) <= {1, 2, 3, 4}
    po = wl["poisson"]
    assert np.array_equal(po["neuron"], np.arange(10)) and np.all(po["rate"] == 0.1)
    if integer:
        assert wl["dtype"] == "i32" and set(np.unique(wl["weight"])) <= {1, 2, 3, 4, 5}
        assert np.all(wl["threshold"] == 10) and np.all(wl["leak"] == 1) and np.all(po["amplitude"] == 11)
    else:
        assert wl["dtype"] == "f32" and np.all((wl["weight"] >= 0) & (wl["weight"] < 1))
        assert np.all(wl["threshold"] == 1) and np.all(wl["leak"] == 0.1) and np.all(po["amplitude"] == 2)
    assert np.all(wl["refractory"] == 2) and np.all(wl["reset"] == 0)


@pytest.mark.parametrize("integer", [False, True])
def test_large_sparse_recipe(integer):
    """Exactly k distinct targets per neuron, delays U{1..16}, the weight
    distribution, thresholds and Poisson inputs of the large sparse network
    (here at 3000 neurons)."""
    n, k = 3000, 100
    wl = W.large_sparse(integer=integer, n=n, k=k)
    pre, post, w, d = wl["pre"], wl["post"], wl["weight"], wl["delay"]
    assert pre.size == n * k and np.all(np.bincount(pre, minlength=n) == k)
    assert np.all(np.diff(pair_keys(pre, post, n)) > 0) and np.all(pre != post)
    assert d.min() == 1 and d.max() == 16 and wl["max_delay"] == 16
    counts = np.bincount(d, minlength=17)[1:]
    assert within(counts.min(), n * k / 16, n * k / 16) and within(counts.max(), n * k / 16, n * k / 16)
    po = wl["poisson"]
    assert po["neuron"].size == n // 100 and np.unique(po["neuron"]).size == n // 100
    assert np.all(po["rate"] == 0.05)
    if integer:
        assert set(np.unique(w)) == set(range(-3, 6))
        assert np.all(wl["threshold"] == 20) and np.all(po["amplitude"] == 21)
    else:
        assert np.all(np.abs(w) >= 1e-3)
        neg = (w < 0).mean()
        assert within(neg * w.size, 0.2 * w.size, w.size * 0.16)
        assert abs(np.abs(w).mean() - 0.5) < 0.01 and abs(np.abs(w).std() - 0.1) < 0.01
        assert np.all((wl["threshold"] >= 0.8) & (wl["threshold"] <= 1.2))
        assert np.all(po["amplitude"] == 2)
    assert np.all(wl["leak"] == (1 if integer else 0.1)) and np.all(wl["refractory"] == 2)


@pytest.mark.parametrize("stdp", [False, True])
def test_large_dense_recipe(stdp):
    n = 512
    wl = W.large_dense(n=n, stdp=stdp)
    w = wl["dense_w"]
    assert w.shape == (n, n) and w.dtype == np.float32
    assert np.all(np.diag(w) == 0)
    off = w[~np.eye(n, dtype=bool)].astype(np.float64)
    assert abs(off.mean()) < 0.02 * 6 / math.sqrt(off.size)
    assert abs(off.std() / 0.02 - 1) < 0.01
    assert wl["dense_delay"] == 1
    po = wl["poisson"]
    assert np.array_equal(po["neuron"], np.arange(n)) and np.all(po["rate"] == 0.02)
    assert np.all(po["amplitude"] == 2)
    assert np.all(wl["threshold"] == 1) and np.all(wl["leak"] == 0.05) and np.all(wl["refractory"] == 1)
    if stdp:
        assert wl["stdp"] == dict(decay=0.9, a_plus=0.01, a_minus=0.012, wmin=-1.0, wmax=1.0)
    else:
        assert wl["stdp"] is None


def test_huge_dense_recipe():
    """sigma = 0.02 sqrt(16384 / n) keeps large-dense's per-step input
    variance (n sigma^2 constant); the device draw has a zero diagonal and
    that spread (drawn here with torch on the CPU)."""
    torch = pytest.importorskip("torch")
    for n in (100_000, 20_000, 16_384):
        wl = W.huge_dense(n=n)
        sig = wl["dense_w_device"]["sigma"]
        assert abs(n * sig * sig - 16384 * 0.02 ** 2) < 1e-12
    wl = W.huge_dense(n=1024)
    w = W.dense_weights_on_device(wl, torch, device="cpu").double().numpy()
    assert w.shape == (1024, 1024) and np.all(np.diag(w) == 0)
    off = w[~np.eye(1024, dtype=bool)]
    assert abs(off.std() / wl["dense_w_device"]["sigma"] - 1) < 0.01
    again = W.dense_weights_on_device(wl, torch, device="cpu").double().numpy()
    assert np.array_equal(w, again)


@pytest.mark.parametrize("n,p", [(100, 0.25), (100, 1.0), (1000, 0.5)])
def test_paper_grid_recipe(n, p):
    """Section 3: Bernoulli(p) digraph, unit weights and delays, three random
    input neurons spiked externally every 10 steps, threshold 1, reset 0,
    refractory 0."""
    wl = W.paper_grid(n, p)
    m = wl["pre"].size
    tot = n * (n - 1)
    assert within(m, p * tot, tot * p * (1 - p))
    assert np.all(wl["weight"] == 1) and np.all(wl["delay"] == 1) and wl["max_delay"] == 1
    ev = wl["events"]
    steps = np.arange(0, 1000, 10)
    assert np.array_equal(ev["step"], np.repeat(steps, 3))
    inputs = ev["neuron"][:3]
    assert np.unique(inputs).size == 3 and np.array_equal(ev["neuron"], np.tile(inputs, steps.size))
    assert np.all(ev["value"] == 2.0)
    assert np.all(wl["threshold"] == 1) and np.all(wl["reset"] == 0) and np.all(wl["refractory"] == 0)
    assert np.all(wl["leak"] == 0)


def test_batched_recipe():
    """Sizes, connection probability, delays, weight scale and Poisson inputs
    of the batched networks follow the recipe; the batch is reproducible and
    a window starting at `first` carries those network indices."""
    nets = W.batched_nets(count=24)
    again = W.batched_nets(count=24)
    for a, b in zip(nets, again):
        for key in ("pre", "post", "weight", "delay", "threshold", "leak", "refractory"):
            assert np.array_equal(a[key], b[key])
    window = W.batched_nets(count=5, first=7)
    assert [wl["net_index"] for wl in window] == list(range(7, 12))
    # the sizes of a window agree with the batch drawn up to its end
    assert [wl["n"] for wl in window] == [wl["n"] for wl in W.batched_nets(count=12)[7:]]
    for wl in nets:
        n, m = wl["n"], wl["pre"].size
        assert 64 <= n <= 4096
        assert np.all(wl["pre"] != wl["post"])
        p_hat = m / (n * (n - 1))
        assert 0.01 - 6 * math.sqrt(0.01 / (n * (n - 1))) <= p_hat <= 0.2 + 6 * math.sqrt(0.2 / (n * (n - 1)))
        assert wl["weight"].dtype == np.float32
        assert set(np.unique(wl["delay"])) <= set(range(1, 9)) and wl["max_delay"] == 8
        # w = N(0, 1) / sqrt(p N): sum of squares over a row is about 1
        if m > 2000:
            assert abs(float((wl["weight"].astype(np.float64) ** 2).sum()) / n - 1) < 0.3
        th = wl["threshold"]
        assert np.all((th >= 0.5) & (th <= 1.5)) and np.all((wl["leak"] >= 0) & (wl["leak"] <= 0.2))
        assert set(np.unique(wl["refractory"])) <= {0, 1, 2, 3}
        po = wl["poisson"]
        assert po["neuron"].size == max(1, n // 10) and np.unique(po["neuron"]).size == po["neuron"].size
        assert np.all(po["amplitude"] == 2.0 * float(np.float32(th).max()))


def test_shared_dense_i8_recipe():
    wl = W.shared_dense_i8(n=256, batch=128, steps=10)
    w = wl["dense_w_i8"]
    assert w.dtype == np.int8 and w.shape == (256, 256)
    assert np.all(np.diag(w) == 0) and w.min() == -8 and w.max() == 8
    off = w[~np.eye(256, dtype=bool)]
    assert set(np.unique(off)) == set(range(-8, 9))
    assert wl["batch"] == 128 and wl["dtype"] == "i32" and wl["dense_delay"] == 1
    assert np.all(wl["threshold"] == 40) and np.all(wl["leak"] == 1) and np.all(wl["refractory"] == 1)
    po = wl["poisson"]
    assert np.array_equal(po["neuron"], np.arange(256)) and np.all(po["rate"] == 0.05)
    assert np.all(po["amplitude"] == 41)


def test_bptt_task_recipe():
    task = W.bptt_task(batch=64, sizes=(300, 200, 10), steps=40)
    x = task["input"]
    assert x.shape == (40, 64, 300) and x.dtype == np.uint8 and set(np.unique(x)) <= {0, 1}
    assert 0.05 < x.mean() < 0.15              # rates U(0, 0.2): mean 0.1
    assert task["labels"].shape == (64,) and task["labels"].min() >= 0 and task["labels"].max() < 10
    for (a, b), w, d in zip([(300, 200), (200, 10)], task["w"], task["delay"]):
        assert w.shape == (a, b) and w.dtype == np.float32
        assert abs(w.astype(np.float64).std() / math.sqrt(2.0 / a) - 1) < 0.1
        assert d.shape == (a, b) and set(np.unique(d)) == {1, 2, 3, 4}
    assert task["checkpoint_every"] == 10 and task["slope"] == 10.0


@pytest.mark.parametrize("make", [
    lambda s: W.tiny(seed=s),
    lambda s: W.large_sparse(n=2000, k=20, seed=s),
    lambda s: W.large_dense(n=256, seed=s),
    lambda s: W.paper_grid(300, 0.25, seed=s),
    lambda s: W.shared_dense_i8(n=128, batch=128, seed=s),
    lambda s: W.random_small(s),
])
def test_seeded_and_deterministic(make):
    """The same seed gives the same arrays; another seed gives others."""
    a, b, c = make(101), make(101), make(202)

    def arrays(wl):
        out = []
        for key in ("pre", "post", "weight", "delay", "dense_w", "dense_w_i8", "threshold"):
            if key in wl:
                out.append(np.asarray(wl[key]))
        out.append(np.asarray(wl["events"]["neuron"]))
        out.append(np.asarray(wl["poisson"]["neuron"]))
        return out

    assert all(np.array_equal(x, y) for x, y in zip(arrays(a), arrays(b)))
    assert not all(x.shape == y.shape and np.array_equal(x, y) for x, y in zip(arrays(a), arrays(c)))
