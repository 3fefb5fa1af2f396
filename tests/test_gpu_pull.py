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


FORMS = [0x1000, 0x2000]     # SN_PULL_PLAIN, SN_PULL_CODED


def run_pull(wl, steps, record=None, form=0):
    S = sn()
    ctx = S.from_workload(wl, flags=S.SN_PROP_PULL | form, record_steps=record or steps)
    assert S.sn_get_propagation(ctx) == S.SN_PULL
    if form:
        assert S.sn_pull_store_info(ctx)[0] == form
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


@pytest.mark.parametrize("form", [0] + FORMS)
@pytest.mark.parametrize("seed", range(12))
def test_random_small_float_bit_exact(seed, form):
    wl = W.random_small(1300 + seed, integer=False, steps=200, events_rate=0.6)
    _, raster, v, r = run_pull(wl, 200, form=form)
    check_float_exact(wl, raster, v, r, 200)


@pytest.mark.parametrize("form", [0] + FORMS)
@pytest.mark.parametrize("seed", range(12))
def test_random_small_int(seed, form):
    wl = W.random_small(1500 + seed, integer=True, steps=200, events_rate=0.6)
    _, raster, v, r = run_pull(wl, 200, form=form)
    compare.check_int_run(wl, raster, v, r, 200)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,D", [(1, 1), (31, 3), (33, 64), (1000, 7), (2049, 16), (40001, 16)])
def test_ragged_sizes_and_delays(n, D, form):
    """Sizes off the 32-neuron slice and the block's chunk; delay 64 (the
    largest) and delay 1 (history of one row)."""
    wl = W.random_small(2100 + n, n=n, integer=False, steps=130, p=min(0.5, 20.0 / n),
                        max_delay=D, events_rate=2.0)
    _, raster, v, r = run_pull(wl, 130, form=form)
    check_float_exact(wl, raster, v, r, 130)
    wi = W.random_small(2200 + n, n=n, integer=True, steps=130, p=min(0.5, 20.0 / n),
                        max_delay=D, events_rate=2.0)
    _, raster, v, r = run_pull(wi, 130, form=form)
    compare.check_int_run(wi, raster, v, r, 130)


@pytest.mark.parametrize("form", FORMS)
def test_duplicate_synapses_keep_input_order(form):
    """Two synapses with the same (delay, pre) add in input order."""
    wl = W.random_small(31, n=40, integer=False, steps=100, p=0.3, max_delay=4, events_rate=3.0)
    k = np.arange(wl["pre"].size)
    for key in ("pre", "post", "delay"):
        wl[key] = np.concatenate([wl[key], wl[key][k[::3]]])
    wl["weight"] = np.concatenate([wl["weight"], (wl["weight"][k[::3]] * 0.37).astype(wl["weight"].dtype)])
    _, raster, v, r = run_pull(wl, 100, form=form)
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


_FULL = {}


@pytest.mark.parametrize("form", [0] + FORMS)
def test_large_sparse_float_full_size_bit_exact(form):
    """N = 100,000, 1e7 synapses, delays 1..16, in the executor the benchmark
    times (the library's choice of store form, then each form forced): every
    spike and the state equal the FP32 mirror's for 120 steps."""
    if "wl" not in _FULL:
        _FULL["wl"] = W.large_sparse(integer=False)
        _FULL["want"] = O.run(_FULL["wl"], O.F32, 120)
    wl = _FULL["wl"]
    st, want, _ = _FULL["want"]
    ctx, raster, v, r = run_pull(wl, 120, form=form)
    assert raster[-1].sum() > 1000
    bad = np.nonzero((raster != want).any(axis=1))[0]
    assert bad.size == 0, f"raster differs first at step {int(bad[0])}"
    assert np.array_equal(np.asarray(v, np.float64), st.v) and np.array_equal(np.asarray(r), st.r)
    S = sn()
    f, nbytes, entries = S.sn_pull_store_info(ctx)
    m = wl["pre"].size
    if form == 0:
        # the library's rule: the plain form while it takes at most 80 % of
        # the L2 (8 bytes a synapse plus padding), else the smaller form
        l2 = torch.cuda.get_device_properties(0).L2_cache_size
        if f == S.SN_PULL_PLAIN:
            assert nbytes <= 0.8 * l2
        else:
            assert 8 * m * 1.5 > 0.8 * l2
    if f == S.SN_PULL_PLAIN:
        assert entries == m and nbytes >= 8 * m
    else:
        # steps above 65,535 (fillers) are rare at 100 synapses a neuron
        assert m <= entries < 1.05 * m and nbytes >= 6 * entries


def gap_network(seed, n, integer, steps):
    """n neurons, three incoming synapses each from uniform pre-neurons with
    uniform delays 1..16, input events at about 20 per step."""
    rng = np.random.default_rng(seed)
    post = np.repeat(np.arange(n, dtype=np.int32), 3)
    pre = ((post + rng.integers(1, n, post.size)) % n).astype(np.int32)
    delay = rng.integers(1, 17, post.size).astype(np.int32)
    if integer:
        w = rng.integers(-2, 6, post.size).astype(np.float64)
        th, lk, rs = np.full(n, 3.0), np.full(n, 1.0), np.zeros(n)
    else:
        w = rng.normal(0.6, 0.5, post.size)
        th, lk, rs = rng.uniform(0.8, 1.2, n), rng.uniform(0.0, 0.1, n), np.zeros(n)
    wl = W._base(n, "i32" if integer else "f32", th, lk, rs, rng.integers(0, 3, n).astype(np.int32), 16, steps)
    order = np.lexsort((post, pre))
    wl.update(pre=pre[order], post=post[order], weight=w[order], delay=delay[order])
    ne = 20 * steps
    val = rng.integers(3, 8, ne).astype(np.float64) if integer else rng.uniform(1.5, 3.0, ne)
    wl["events"] = dict(step=rng.integers(0, steps, ne).astype(np.int32),
                        neuron=rng.integers(0, n, ne).astype(np.int32), value=val)
    wl["name"] = f"gap-network-{seed}"
    return wl


@pytest.mark.parametrize("integer", [False, True])
def test_coded_store_gap_fillers(integer):
    """70,000 neurons with three incoming synapses each over delays 1..16: the
    steps between a neuron's bit offsets are mostly above 65,535, so the coded
    store holds many filler entries (weight 0, bit tests anywhere in the
    window).  Both forms give the oracle's run bit for bit."""
    S = sn()
    n, steps = 70_000, 130
    wl = gap_network(4242 + integer, n, integer, steps)
    st, want, _ = O.run(wl, O.INT if integer else O.F32, steps)
    assert want[20:].sum() > 100
    infos = {}
    for form in FORMS:
        ctx, raster, v, r = run_pull(wl, steps, form=form)
        infos[form] = S.sn_pull_store_info(ctx)
        bad = np.nonzero((raster != want).any(axis=1))[0]
        assert bad.size == 0, f"form {form:#x}: raster differs first at step {int(bad[0])}"
        assert np.array_equal(np.asarray(v, np.float64), st.v) and np.array_equal(np.asarray(r), st.r)
    m = wl["pre"].size
    assert infos[FORMS[0]][2] == m
    assert infos[FORMS[1]][2] > 2 * m          # fillers
    # the library's own choice is the smaller store: here the plain one
    ctx = S.from_workload(wl, flags=S.SN_PROP_PULL, record_steps=4)
    assert S.sn_pull_store_info(ctx)[0] == S.SN_PULL_PLAIN


def test_pull_store_info_before_and_after_build():
    S = sn()
    wl = W.random_small(77, n=300, integer=True, steps=10)
    ctx = S.from_workload(wl, record_steps=10)
    assert S.sn_pull_store_info(ctx) == (0, 0, 0)
    S.sn_set_propagation(ctx, S.SN_PULL)
    f, nbytes, entries = S.sn_pull_store_info(ctx)
    assert f in (S.SN_PULL_PLAIN, S.SN_PULL_CODED) and entries >= wl["pre"].size and nbytes > 0


def test_large_sparse_int_full_size():
    wl = W.large_sparse(integer=True)
    _, raster, v, r = run_pull(wl, 150)
    assert raster.sum() > 0
    compare.check_int_run(wl, raster, v, r, 150)
