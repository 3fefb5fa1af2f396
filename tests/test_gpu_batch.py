"""Batched simulation of many independent networks in one persistent launch:
parity of every network with the oracle (integer: bit-exact; float: the
comparison rules), independence of the executor mapping, equality with the
plain single-network path, and sampled networks of the full 4096-network
configuration."""

import numpy as np
import pytest

from oracle import compare, oracle as O
from paper_2305_02510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def S():
    from paper_2305_02510_gb300 import sn
    return sn


def run_batch(nets, steps, config=None, tune=False):
    s = S()
    ctx = s.from_batch_workloads(nets, record_steps=steps)
    if config is not None:
        s.sn_batch_config(ctx, *config)
    if tune:
        s.sn_autotune(ctx, 5)
    s.sn_run(ctx, steps)
    s.sn_sync(ctx)
    rasters = s.split_batch_raster(s.sn_get_spikes(ctx, 0, steps), ctx.net_n)
    v, r = s.sn_get_state(ctx)
    off = np.cumsum([0] + ctx.net_n)
    return ctx, rasters, [v[off[b]:off[b + 1]] for b in range(len(nets))], \
        [r[off[b]:off[b + 1]] for b in range(len(nets))]


def int_nets(count, seed=0):
    nets = []
    for k in range(count):
        n = [3, 17, 31, 32, 33, 64, 100, 129, 257, 300, 513, 700, 1025, 2000, 4096][k % 15]
        wl = W.random_small(5000 + seed * 100 + k, n=n, integer=True, steps=150,
                            p=min(0.5, 12.0 / n), max_delay=1 + k % 8, events_rate=1.5)
        wl["poisson"] = dict(neuron=np.arange(0, n, 7, dtype=np.int32), rate=np.full((n + 6) // 7, 0.05),
                             amplitude=np.full((n + 6) // 7, 9.0), seed=77)
        nets.append(wl)
    return nets


@pytest.mark.parametrize("config", [(0, 0), (512, 0), (128, 96 * 1024), (512, 176 * 1024), (64, 32 * 1024)])
def test_batch_int_bit_exact(config):
    nets = int_nets(30)
    _, rasters, vs, rs = run_batch(nets, 150, config)
    for b, wl in enumerate(nets):
        st, want, _ = O.run(wl, O.INT, 150, net_index=b, poisson_seed=77)
        assert np.array_equal(rasters[b], want), f"net {b} (n={wl['n']})"
        assert np.array_equal(vs[b].astype(np.float64), st.v) and np.array_equal(rs[b], st.r)


def test_batch_float_small_sample():
    nets = W.batched_nets(count=40, steps=200)
    _, rasters, vs, rs = run_batch(nets, 200, tune=True)
    for b, wl in enumerate(nets):
        compare.check_float_run(wl, rasters[b], vs[b], rs[b], 200, net_index=b)


def test_batch_equals_plain_single_contexts():
    """Fixed-point accumulation makes the batched and the single-network
    executors bit-identical on the same network and input stream."""
    s = S()
    nets = W.batched_nets(count=12, steps=120)
    _, rasters, vs, rs = run_batch(nets, 120)
    for b, wl in enumerate(nets):
        ctx = s.sn_create(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], wl["pre"], wl["post"],
                          wl["weight"], wl["delay"], max_delay=8, record_steps=120)
        po = wl["poisson"]
        s.sn_set_poisson_stream(ctx, po["neuron"], po["rate"], po["amplitude"], po["seed"], b)
        s.sn_run(ctx, 120)
        got = s.unpack_raster(s.sn_get_spikes(ctx, 0, 120), wl["n"])
        v, r = s.sn_get_state(ctx)
        assert np.array_equal(got, rasters[b]) and np.array_equal(v, vs[b]) and np.array_equal(r, rs[b])


def test_batch_resume_across_runs():
    s = S()
    nets = int_nets(15, seed=3)
    ctx = s.from_batch_workloads(nets, record_steps=150)
    for k in (40, 0, 1, 109):
        s.sn_run(ctx, k)
    rasters = s.split_batch_raster(s.sn_get_spikes(ctx, 0, 150), ctx.net_n)
    for b, wl in enumerate(nets):
        _, want, _ = O.run(wl, O.INT, 150, net_index=b, poisson_seed=77)
        assert np.array_equal(rasters[b], want)
    steps, spikes, events = s.sn_get_counters(ctx)
    assert steps == 150 and spikes == sum(int(x.sum()) for x in rasters)


def test_batch_full_size_sampled():
    """The 4096-network, 500-step configuration in one persistent launch
    (autotuned mapping); 10 networks across the size range checked against
    the oracle."""
    s = S()
    nets = W.batched_nets(count=4096, steps=500)
    ctx = s.from_batch_workloads(nets, record_steps=500)
    s.sn_autotune(ctx, 10)
    s.sn_run(ctx, 500)
    s.sn_sync(ctx)
    bits = s.sn_get_spikes(ctx, 0, 500)
    v, r = s.sn_get_state(ctx)
    order = np.argsort([w["n"] for w in nets])
    pick = [int(order[k]) for k in np.linspace(0, len(nets) - 1, 10).astype(int)]
    off = np.cumsum([0] + ctx.net_n)
    woff = np.cumsum([0] + [(n + 31) // 32 for n in ctx.net_n])
    for b in pick:
        wl = nets[b]
        got = s.unpack_raster(np.ascontiguousarray(bits[:, woff[b]:woff[b + 1]]), wl["n"])
        compare.check_float_run(wl, got, v[off[b]:off[b + 1]], r[off[b]:off[b + 1]], 500, net_index=b)


@pytest.mark.parametrize("kind", ["int", "float"])
def test_batch_checkpoint_resume_bit_exact(kind):
    """run(T) equals run(T1); save; load into a fresh context; run(T - T1):
    every network's spikes, state and the counters."""
    s = S()
    nets = int_nets(20, seed=3) if kind == "int" else W.batched_nets(count=24, steps=150)
    T, T1 = 150, 61
    ctx = s.from_batch_workloads(nets, record_steps=T)
    s.sn_run(ctx, T)
    want = s.sn_get_spikes(ctx, 0, T)
    v_want, r_want = s.sn_get_state(ctx)
    a = s.from_batch_workloads(nets, record_steps=T)
    s.sn_run(a, T1)
    first = s.sn_get_spikes(a, 0, T1)
    blob = s.sn_save(a)
    b = s.from_batch_workloads(nets, record_steps=T)
    s.sn_load(b, blob)
    s.sn_run(b, T - T1)
    second = s.sn_get_spikes(b, T1, T)
    v, r = s.sn_get_state(b)
    assert np.array_equal(np.concatenate([first, second]), want)
    assert np.array_equal(v, v_want) and np.array_equal(r, r_want)
    assert tuple(s.sn_get_counters(b)) == tuple(s.sn_get_counters(ctx))
    # a checkpoint of another set of networks is refused
    other = s.from_batch_workloads(nets[:-1], record_steps=T)
    with pytest.raises(s.SnError):
        s.sn_load(other, blob)
