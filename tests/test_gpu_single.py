"""Parity of the CUDA single-network path (sparse push, dense gather, STDP)
with the CPU oracle, through the C ABI.

Integer networks: bit-exact rasters and states.  Float networks: the rules in
oracle/compare.py (spikes equal except at near-threshold states, states
within 1e-5 of max(|V|, |theta|), teacher-forced steps after a divergence).
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


EXEC = {"cta": 1, "grid": 2}


def run_gpu(wl, steps, flags=0, record=None):
    S = sn()
    ctx = S.from_workload(wl, flags=flags, record_steps=record or steps)
    S.sn_run(ctx, steps)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, steps), wl["n"])
    v, r = S.sn_get_state(ctx)
    return ctx, raster, v, r


def segments(wl, points, flags=0):
    """Run the simulator and capture, for each t in points, the state after
    step t-1, the spike rows t-D..t-1, and step t's spikes and state."""
    S = sn()
    last = max(points) + 1
    ctx = S.from_workload(wl, flags=flags, record_steps=last)
    D = wl["max_delay"]
    out = []
    done = 0
    for t in sorted(points):
        S.sn_run(ctx, t - done)
        v0, r0 = S.sn_get_state(ctx)
        x0 = S.sn_get_trace(ctx) if wl.get("stdp") else None
        w0 = S.sn_get_weights(ctx) if wl.get("stdp") else None
        S.sn_run(ctx, 1)
        v1, r1 = S.sn_get_state(ctx)
        x1 = S.sn_get_trace(ctx) if wl.get("stdp") else None
        w1 = S.sn_get_weights(ctx) if wl.get("stdp") else None
        rows = S.unpack_raster(S.sn_get_spikes(ctx, max(0, t - D), t + 1), wl["n"])
        hist = np.zeros((D, wl["n"]), np.uint8)
        hist[D - (rows.shape[0] - 1):] = rows[:-1]
        out.append(dict(t=t, v0=v0, r0=r0, hist=hist, row=rows[-1], v1=v1, r1=r1,
                        x0=x0, x1=x1, w0=w0, w1=w1))
        done = t + 1
    return ctx, out


def teacher(wl, seg, mode):
    n = 0
    for s in seg:
        n += compare.teacher_forced_step(wl, s["t"], s["v0"], s["r0"], s["hist"], s["row"], s["v1"],
                                         s["r1"], mode, trace_prev=s["x0"], w_prev=s["w0"],
                                         w=s["w1"], trace=s["x1"])
    return n


@pytest.mark.parametrize("ex", ["cta", "grid"])
def test_tiny_int_bit_exact(ex):
    wl = W.tiny(integer=True)
    _, raster, v, r = run_gpu(wl, 1000, EXEC[ex])
    assert raster.sum() > 100
    compare.check_int_run(wl, raster, v, r, 1000)


@pytest.mark.parametrize("ex", ["cta", "grid"])
def test_tiny_float(ex):
    wl = W.tiny(integer=False)
    _, raster, v, r = run_gpu(wl, 1000, EXEC[ex])
    first, _ = compare.check_float_run(wl, raster, v, r, 1000)
    _, seg = segments(wl, [1, 250, 500, 999], EXEC[ex])
    teacher(wl, seg, O.F32)


@pytest.mark.parametrize("seed", range(24))
def test_random_small_int(seed):
    wl = W.random_small(500 + seed, integer=True, steps=200, events_rate=0.6)
    _, raster, v, r = run_gpu(wl, 200, EXEC["cta" if seed % 2 else "grid"])
    compare.check_int_run(wl, raster, v, r, 200)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_float(seed):
    wl = W.random_small(700 + seed, integer=False, steps=200, events_rate=0.6)
    _, raster, v, r = run_gpu(wl, 200, EXEC["cta" if seed % 2 else "grid"])
    compare.check_float_run(wl, raster, v, r, 200)


@pytest.mark.parametrize("n", [1, 31, 33, 1000, 2049, 5000, 40001])
def test_ragged_sizes_int(n):
    """Sizes that are not multiples of the 32-neuron raster word or of a
    block's chunk, on the grid executor (and the one-block one when small)."""
    wl = W.random_small(900 + n, n=n, integer=True, steps=120, p=min(0.5, 20.0 / n),
                        max_delay=5, events_rate=2.0)
    _, raster, v, r = run_gpu(wl, 120, EXEC["grid"])
    compare.check_int_run(wl, raster, v, r, 120)
    if n <= 5000:
        _, raster, v, r = run_gpu(wl, 120, EXEC["cta"])
        compare.check_int_run(wl, raster, v, r, 120)


def test_no_synapses_and_no_input():
    wl = W.random_small(17, n=50, integer=True, steps=30, p=0.0)
    assert wl["pre"].size == 0
    _, raster, v, r = run_gpu(wl, 30)
    compare.check_int_run(wl, raster, v, r, 30)
    wl["events"] = dict(step=np.zeros(0, np.int32), neuron=np.zeros(0, np.int32), value=np.zeros(0))
    _, raster, v, r = run_gpu(wl, 30)
    assert raster.sum() == 0


def test_zero_steps_and_resume():
    S = sn()
    wl = W.tiny(integer=True)
    ctx = S.from_workload(wl, record_steps=400)
    S.sn_run(ctx, 0)
    for k in (150, 1, 0, 249):
        S.sn_run(ctx, k)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 400), wl["n"])
    v, r = S.sn_get_state(ctx)
    compare.check_int_run(wl, raster, v, r, 400)
    steps, spikes, events = S.sn_get_counters(ctx)
    assert steps == 400 and spikes == raster.sum()
    deg = np.bincount(wl["pre"], minlength=wl["n"])
    assert events == int((raster * deg[None, :]).sum())


@pytest.mark.parametrize("kind", ["int", "float", "dense-stdp"])
def test_checkpoint_resume_bit_exact(kind):
    """run(T) equals run(T1); save; load into a fresh context; run(T - T1)."""
    S = sn()
    if kind == "dense-stdp":
        wl = W.large_dense(n=1024, stdp=True, steps=200)
    else:
        wl = W.tiny(integer=kind == "int")
    T, T1 = 200, 77
    ctx = S.from_workload(wl, record_steps=T)
    S.sn_run(ctx, T)
    want = S.unpack_raster(S.sn_get_spikes(ctx, 0, T), wl["n"])
    v_want, r_want = S.sn_get_state(ctx)
    a = S.from_workload(wl, record_steps=T)
    S.sn_run(a, T1)
    blob = S.sn_save(a)
    first = S.unpack_raster(S.sn_get_spikes(a, 0, T1), wl["n"])
    b = S.from_workload(wl, record_steps=T)
    S.sn_load(b, blob)
    S.sn_run(b, T - T1)
    second = S.unpack_raster(S.sn_get_spikes(b, T1, T), wl["n"])
    v, r = S.sn_get_state(b)
    assert np.array_equal(np.concatenate([first, second]), want)
    assert np.array_equal(v, v_want) and np.array_equal(r, r_want)
    if kind == "dense-stdp":
        assert np.array_equal(S.sn_get_weights(b), S.sn_get_weights(ctx))


def test_large_sparse_int_full_size():
    """N = 100,000, 1e7 synapses, delays 1..16: raster and state bit-exact
    for 250 steps, then teacher-forced steps up to step 999."""
    wl = W.large_sparse(integer=True)
    T0 = 250
    ctx, raster, v, r = run_gpu(wl, T0, record=1000)
    assert raster.sum() > 0
    compare.check_int_run(wl, raster, v, r, T0)
    _, seg = segments(wl, [400, 999])
    teacher(wl, seg, O.INT)


def test_large_sparse_float_full_size():
    wl = W.large_sparse(integer=False)
    T0 = 60
    _, raster, v, r = run_gpu(wl, T0)
    compare.check_float_run(wl, raster, v, r, T0)
    _, seg = segments(wl, [100, 500, 999])
    assert teacher(wl, seg, O.F32) > 1000


@pytest.mark.parametrize("stdp", [False, True])
def test_dense_medium(stdp):
    wl = W.large_dense(n=2000, stdp=stdp, steps=300)
    _, raster, v, r = run_gpu(wl, 300)
    assert raster.sum() > 0
    compare.check_float_run(wl, raster, v, r, 300)
    _, seg = segments(wl, [0, 1, 150, 299])
    teacher(wl, seg, O.F32)


def test_dense_ragged_and_delay():
    """Dense net with n not a multiple of 4 or 32 and a dense delay of 3."""
    wl = W.large_dense(n=333, steps=200)
    wl["dense_delay"] = 3
    wl["max_delay"] = 4
    _, raster, v, r = run_gpu(wl, 200)
    compare.check_float_run(wl, raster, v, r, 200)


@pytest.mark.parametrize("stdp", [False, True])
def test_dense_full_size_teacher_forced(stdp):
    """N = 16384 all-to-all (1 GiB of weights): teacher-forced steps."""
    wl = W.large_dense(stdp=stdp, steps=1000)
    _, seg = segments(wl, [3, 400])
    assert teacher(wl, seg, O.F32) > 100


def test_sparse_stdp_tiny():
    """STDP on a sparse net (all delays 1): bit-identical weights while the
    spikes agree."""
    wl = W.random_small(4242, n=60, integer=False, steps=150, max_delay=1, p=0.2,
                        events_rate=1.5)
    wl["stdp"] = dict(decay=0.9, a_plus=0.01, a_minus=0.012, wmin=-1.0, wmax=1.0)
    S = sn()
    ctx, raster, v, r = run_gpu(wl, 150)
    first, st = compare.check_float_run(wl, raster, v, r, 150)
    if first is None:
        assert np.array_equal(S.sn_get_weights(ctx).astype(np.float64), st.w)
        assert np.array_equal(S.sn_get_trace(ctx).astype(np.float64), st.trace)
    _, seg = segments(wl, [5, 77, 149])
    teacher(wl, seg, O.F32)


def test_integer_overflow_is_reported():
    """An integer state that leaves the int32 range latches SN_EOVERFLOW; the
    context then refuses to run."""
    S = sn()
    n = 4
    ctx = S.sn_create(np.full(n, np.inf), np.zeros(n), np.zeros(n), np.zeros(n, np.int32),
                      np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0, np.int32),
                      dtype=S.SN_I32, max_delay=1)
    S.sn_set_input(ctx, np.arange(300, dtype=np.int32), np.zeros(300, np.int32),
                   np.full(300, 2.0**23 - 1))
    S.sn_run(ctx, 200)
    S.sn_sync(ctx)                      # 200 * (2^23 - 1) < 2^31: fine
    v, _ = S.sn_get_state(ctx)
    assert v[0] == 200 * (2**23 - 1)
    S.sn_run(ctx, 100)
    with pytest.raises(S.SnError) as e:
        S.sn_sync(ctx)
    assert e.value.status == S.SN_EOVERFLOW
    with pytest.raises(S.SnError) as e:
        S.sn_run(ctx, 1)
    assert e.value.status == S.SN_ESTATE
