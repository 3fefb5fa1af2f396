"""Pull propagation of sparse networks through the C ABI, against the CPU
oracle.

Pull sums each neuron's incoming weights in float, the oldest spikes first
(descending delay, then ascending pre and input index), the order of the
oracle's FP32 mirror, so float runs must match the mirror bit for bit (spikes
and states, every step), not only within the float tolerance; integer runs are bit-exact as always.  Switching between
push and pull, checkpoints across the switch and the autotuner's choice must
leave the trajectory unchanged.
"""

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


def sn():
    from paper_2305_02510_gb300 import sn as m
    return m


def run_pull(wl, steps, record=None):
    S = sn()
    ctx = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=record or steps)
    assert S.sn_get_propagation(ctx) == S.SN_PULL
    S.sn_run(ctx, steps)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, steps), wl["n"])
    v, r = S.sn_get_state(ctx)
    return ctx, raster, v, r


def check_float_exact(wl, raster, v, r, steps):
    """Spikes of every step and the final state equal the FP32 mirror's."""
    st, want, _ = O.run(wl, O.F32, steps)
    bad = np.nonzero((raster != want).any(axis=1))[0]
    assert bad.size == 0, f"raster differs first at step {int(bad[0])}"
    vv = np.asarray(v, np.float32)
    assert np.array_equal(vv.astype(np.float64), st.v), \
        f"state differs at neurons {np.nonzero(vv.astype(np.float64) != st.v)[0][:8].tolist()}"
    assert np.array_equal(np.asarray(r), st.r)
    return st


def test_tiny_float_bit_exact():
    wl = W.tiny(integer=False)
    _, raster, v, r = run_pull(wl, 1000)
    assert raster.sum() > 100
    check_float_exact(wl, raster, v, r, 1000)


def test_tiny_int_bit_exact():
    wl = W.tiny(integer=True)
    _, raster, v, r = run_pull(wl, 1000)
    compare.check_int_run(wl, raster, v, r, 1000)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_float_bit_exact(seed):
    wl = W.random_small(1300 + seed, integer=False, steps=200, events_rate=0.6)
    _, raster, v, r = run_pull(wl, 200)
    check_float_exact(wl, raster, v, r, 200)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_int(seed):
    wl = W.random_small(1500 + seed, integer=True, steps=200, events_rate=0.6)
    _, raster, v, r = run_pull(wl, 200)
    compare.check_int_run(wl, raster, v, r, 200)


@pytest.mark.parametrize("n,D", [(1, 1), (31, 3), (33, 64), (1000, 7), (2049, 16), (40001, 16)])
def test_ragged_sizes_and_delays(n, D):
    """Sizes off the 32-neuron slice and the block's chunk; delay 64 (the
    largest) and delay 1 (history of one row)."""
    wl = W.random_small(2100 + n, n=n, integer=False, steps=130, p=min(0.5, 20.0 / n),
                        max_delay=D, events_rate=2.0)
    _, raster, v, r = run_pull(wl, 130)
    check_float_exact(wl, raster, v, r, 130)
    wi = W.random_small(2200 + n, n=n, integer=True, steps=130, p=min(0.5, 20.0 / n),
                        max_delay=D, events_rate=2.0)
    _, raster, v, r = run_pull(wi, 130)
    compare.check_int_run(wi, raster, v, r, 130)


def test_duplicate_synapses_keep_input_order():
    """Two synapses with the same (delay, pre) add in input order."""
    wl = W.random_small(31, n=40, integer=False, steps=100, p=0.3, max_delay=4, events_rate=3.0)
    k = np.arange(wl["pre"].size)
    for key in ("pre", "post", "delay"):
        wl[key] = np.concatenate([wl[key], wl[key][k[::3]]])
    wl["weight"] = np.concatenate([wl["weight"], (wl["weight"][k[::3]] * 0.37).astype(wl["weight"].dtype)])
    _, raster, v, r = run_pull(wl, 100)
    check_float_exact(wl, raster, v, r, 100)


def test_no_synapses_and_zero_steps():
    S = sn()
    wl = W.random_small(17, n=50, integer=True, steps=30, p=0.0)
    ctx = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=30)
    S.sn_run(ctx, 0)
    for k in (11, 0, 19):
        S.sn_run(ctx, k)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 30), wl["n"])
    v, r = S.sn_get_state(ctx)
    compare.check_int_run(wl, raster, v, r, 30)


@pytest.mark.parametrize("integer", [True, False])
def test_switching_push_and_pull(integer):
    """push 40, pull 55, push 1, pull 70, push 34: pending input crosses each
    switch (delays up to 8).  Integer: bit-exact.  Float: the push segments
    round differently, so the float rules apply."""
    S = sn()
    wl = W.random_small(77, n=300, integer=integer, steps=200, p=0.08, max_delay=8, events_rate=2.0)
    ctx = S.from_workload(wl, record_steps=200)
    for mode, k in ((S.SN_PUSH, 40), (S.SN_PULL, 55), (S.SN_PUSH, 1), (S.SN_PULL, 70), (S.SN_PUSH, 34)):
        S.sn_set_propagation(ctx, mode)
        S.sn_run(ctx, k)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 200), wl["n"])
    v, r = S.sn_get_state(ctx)
    assert raster.sum() > 50
    if integer:
        compare.check_int_run(wl, raster, v, r, 200)
    else:
        compare.check_float_run(wl, raster, v, r, 200)
    steps, spikes, events = S.sn_get_counters(ctx)
    deg = np.bincount(wl["pre"], minlength=wl["n"])
    assert steps == 200 and spikes == raster.sum() and events == int((raster * deg[None, :]).sum())


@pytest.mark.parametrize("resume", ["pull", "push"])
def test_checkpoint_of_pull_run(resume):
    """run(T) with pull equals pull run(T1); save; load into a fresh context
    (pull or push); run(T - T1).  The checkpoint carries the spikes whose
    deliveries are still due."""
    S = sn()
    wl = W.random_small(91, n=500, integer=True, steps=200, p=0.05, max_delay=12, events_rate=2.0)
    T, T1 = 200, 83
    _, want, v_want, r_want = run_pull(wl, T)
    a = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=T)
    S.sn_run(a, T1)
    blob = S.sn_save(a)
    first = S.unpack_raster(S.sn_get_spikes(a, 0, T1), wl["n"])
    b = S.from_workload(wl, flags=S.SN_PROP_PULL if resume == "pull" else 0, record_steps=T)
    S.sn_load(b, blob)
    S.sn_run(b, T - T1)
    second = S.unpack_raster(S.sn_get_spikes(b, T1, T), wl["n"])
    v, r = S.sn_get_state(b)
    assert np.array_equal(np.concatenate([first, second]), want)
    assert np.array_equal(v, v_want) and np.array_equal(r, r_want)


def test_float_checkpoint_pull_bit_exact():
    S = sn()
    wl = W.random_small(93, n=700, integer=False, steps=150, p=0.03, max_delay=6, events_rate=2.0)
    T, T1 = 150, 64
    _, want, v_want, _ = run_pull(wl, T)
    a = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=T)
    S.sn_run(a, T1)
    blob = S.sn_save(a)
    b = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=T)
    S.sn_load(b, blob)
    S.sn_run(b, T - T1)
    second = S.unpack_raster(S.sn_get_spikes(b, T1, T), wl["n"])
    v, _ = S.sn_get_state(b)
    assert np.array_equal(second, want[T1:])
    assert np.array_equal(np.asarray(v).view(np.uint32), np.asarray(v_want).view(np.uint32))


def test_autotune_then_exact():
    S = sn()
    wl = W.random_small(55, n=3000, integer=True, steps=150, p=0.01, max_delay=9, events_rate=2.0)
    ctx = S.from_workload(wl, record_steps=150)
    ms = S.sn_autotune(ctx, 20)
    assert ms > 0
    assert S.sn_get_propagation(ctx) in (S.SN_PUSH, S.SN_PULL)
    S.sn_run(ctx, 150)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 150), wl["n"])
    v, r = S.sn_get_state(ctx)
    compare.check_int_run(wl, raster, v, r, 150)


def test_unsupported_cases():
    S = sn()
    wl = W.large_dense(n=64, stdp=True, steps=10)
    dense = S.from_workload(wl)
    with pytest.raises(S.SnError) as e:
        S.sn_set_propagation(dense, S.SN_PULL)
    assert e.value.status == S.SN_EUNSUPPORTED
    # STDP runs on push
    ws = W.random_small(5, n=64, integer=False, steps=10, p=0.1, max_delay=1)
    ctx = S.from_workload(ws, flags=S.SN_PROP_PULL)
    S.sn_stdp(ctx, 0.9, 0.01, 0.012, -1.0, 1.0, True)
    assert S.sn_get_propagation(ctx) == S.SN_PUSH
    with pytest.raises(S.SnError) as e:
        S.sn_set_propagation(ctx, S.SN_PULL)
    assert e.value.status == S.SN_EUNSUPPORTED
    # a history of 64 steps x 200,000 neurons does not fit a block's shared memory
    n = 200000
    with pytest.raises(S.SnError) as e:
        S.sn_create(np.ones(n), np.zeros(n), np.zeros(n), np.zeros(n, np.int32), np.zeros(0, np.int32),
                    np.zeros(0, np.int32), np.zeros(0), np.zeros(0, np.int32), dtype=S.SN_I32,
                    max_delay=64, flags=S.SN_PROP_PULL)
    assert e.value.status == S.SN_EUNSUPPORTED


def test_large_sparse_float_full_size_bit_exact():
    """N = 100,000, 1e7 synapses, delays 1..16, in the executor the benchmark
    times: every spike and the state equal the FP32 mirror's for 120 steps."""
    wl = W.large_sparse(integer=False)
    _, raster, v, r = run_pull(wl, 120)
    assert raster[-1].sum() > 1000
    check_float_exact(wl, raster, v, r, 120)


def test_large_sparse_int_full_size():
    wl = W.large_sparse(integer=True)
    _, raster, v, r = run_pull(wl, 150)
    assert raster.sum() > 0
    compare.check_int_run(wl, raster, v, r, 150)
