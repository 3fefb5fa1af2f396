"""Wide column slabs of the dense executor, checked over long single launches.

The dense kernel gives each block a slab of 32 * k weight columns; k = 1 up to
about 19,000 neurons, and 2, 4 and 8 only beyond (8 for the 100,000-neuron
network).  SN_DENSE_SLAB(k) forces the slab width, so networks small enough
for a full oracle run take the wide-slab code, and every step of a launch of
hundreds of steps (the ring, the two-row spike buffer and the slab's partial
sums inside one persistent launch) is compared with the oracle:
  - integer-valued weights (workloads.dense_integer_valued): every sum is
    exact in float32, so rasters and states equal the oracle's bit for bit;
  - N(0, sigma) weights, with and without STDP: the float rules of
    oracle/compare.py, then teacher-forced steps.
n % 4 != 0 takes the scalar gather, n % 4 == 0 the vector gather."""

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


def run_one_launch(wl, steps, k):
    """One sn_run of `steps` steps with the slab width forced to 32 * k."""
    from paper_2305_02510_gb300 import sn as S
    ctx = S.from_workload(wl, flags=S.SN_DENSE_SLAB(k), record_steps=steps)
    S.sn_run(ctx, steps)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, steps), wl["n"])
    v, r = S.sn_get_state(ctx)
    return ctx, raster, v, r


_ORACLE = {}


def integer_case(n, steps):
    """The integer-valued network of n neurons and its oracle run (computed
    once per size for all slab widths)."""
    if n not in _ORACLE:
        wl = W.dense_integer_valued(n, steps=steps)
        st, want, _ = O.run(wl, O.F32, steps)
        _ORACLE[n] = (wl, st, want)
    return _ORACLE[n]


@pytest.mark.parametrize("k", [1, 2, 4, 8])
@pytest.mark.parametrize("n", [2000, 3001, 4999])
def test_integer_valued_one_launch_bit_exact(n, k):
    steps = 250
    wl, st, want = integer_case(n, steps)
    ctx, raster, v, r = run_one_launch(wl, steps, k)
    bad = np.nonzero((raster != want).any(axis=1))[0]
    assert bad.size == 0, f"slab {32 * k}: raster differs first at step {int(bad[0])}"
    assert np.array_equal(np.asarray(v, np.float64), st.v)
    assert np.array_equal(np.asarray(r), st.r)
    # most spikes come through synapses, not only from the Poisson input
    assert want[100:].mean() > 0.05
    from paper_2305_02510_gb300 import sn as S
    steps_done, spikes, events = S.sn_get_counters(ctx)
    assert steps_done == steps and spikes == int(want.sum()) and events == spikes * n


@pytest.mark.parametrize("k", [2, 4, 8])
@pytest.mark.parametrize("n", [2000, 2001])
def test_float_one_launch(n, k):
    steps = 300
    wl = W.large_dense(n=n, steps=steps)
    _, raster, v, r = run_one_launch(wl, steps, k)
    assert raster.sum() > 0
    compare.check_float_run(wl, raster, v, r, steps)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_stdp_one_launch(k):
    """STDP in wide slabs: the float rules over a 300-step launch, then
    teacher-forced steps with the weights and traces in between."""
    from paper_2305_02510_gb300 import sn as S
    steps = 300
    wl = W.large_dense(n=2000, stdp=True, steps=steps)
    _, raster, v, r = run_one_launch(wl, steps, k)
    assert raster.sum() > 0
    compare.check_float_run(wl, raster, v, r, steps)
    ctx = S.from_workload(wl, flags=S.SN_DENSE_SLAB(k), record_steps=steps)
    done, checked = 0, 0
    for t in (1, 120, 299):
        S.sn_run(ctx, t - done)
        v0, r0 = S.sn_get_state(ctx)
        x0, w0 = S.sn_get_trace(ctx), S.sn_get_weights(ctx)
        prev = S.unpack_raster(S.sn_get_spikes(ctx, t - 1, t + 0), wl["n"])
        S.sn_run(ctx, 1)
        v1, r1 = S.sn_get_state(ctx)
        x1, w1 = S.sn_get_trace(ctx), S.sn_get_weights(ctx)
        row = S.unpack_raster(S.sn_get_spikes(ctx, t, t + 1), wl["n"])[0]
        checked += compare.teacher_forced_step(wl, t, v0, r0, prev, row, v1, r1, O.F32,
                                               trace_prev=x0, w_prev=w0, w=w1, trace=x1)
        done = t + 1
    assert checked > 0


def test_slab_widths_give_equal_integer_runs():
    """The four slab widths on one integer-valued network: identical rasters
    and states (every sum exact)."""
    steps, n = 200, 1536
    wl = W.dense_integer_valued(n, steps=steps)
    runs = [run_one_launch(wl, steps, k)[1:] for k in (1, 2, 4, 8)]
    for raster, v, r in runs[1:]:
        assert np.array_equal(raster, runs[0][0])
        assert np.array_equal(v, runs[0][1]) and np.array_equal(r, runs[0][2])


def test_forced_slab_arguments():
    from paper_2305_02510_gb300 import sn as S
    wl = W.large_dense(n=64, steps=4)
    with pytest.raises(S.SnError) as e:
        S.from_workload(wl, flags=S.SN_DENSE_SLAB(3))
    assert e.value.status == S.SN_EINVAL
