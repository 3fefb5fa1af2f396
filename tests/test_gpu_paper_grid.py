"""The paper's benchmark networks (Section 3, Table 2): Bernoulli(p) digraphs
with unit weights and delays, threshold 1, reset 0, no refractory period and
three input neurons spiked every 10 steps.  Every sum is a small integer, so
the float32 simulation is exact: rasters and states must equal the oracle's
bit for bit, on the dense path (sn_create_dense) and on both propagation
modes of the sparse path (sn_create).
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_02510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def dense_of(wl):
    w = np.zeros((wl["n"], wl["n"]), np.float32)
    w[wl["pre"], wl["post"]] = 1.0
    return w


def run(wl, steps, how):
    from paper_2305_02510_gb300 import sn as S
    if how == "dense":
        ctx = S.sn_create_dense(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], dense_of(wl), 1,
                                max_delay=1, record_steps=steps)
        ev = wl["events"]
        S.sn_set_input(ctx, ev["step"], ev["neuron"], ev["value"])
    else:
        ctx = S.from_workload(wl, record_steps=steps)
        try:
            S.sn_set_propagation(ctx, S.SN_PULL if how == "pull" else S.SN_PUSH)
        except S.SnError as e:
            assert e.status == S.SN_EUNSUPPORTED
            pytest.skip("pull does not fit this network")
    S.sn_run(ctx, steps)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, steps), wl["n"])
    v, r = S.sn_get_state(ctx)
    _, _, ev = S.sn_get_counters(ctx)
    return raster, v, r, ev


@pytest.mark.parametrize("how", ["dense", "push", "pull"])
@pytest.mark.parametrize("n,p", [(100, 0.25), (100, 1.0), (1000, 0.25), (1000, 0.5), (1000, 0.75),
                                 (1000, 1.0)])
def test_paper_grid_exact(n, p, how):
    steps = 120
    wl = W.paper_grid(n, p, steps=steps)
    raster, v, r, ev = run(wl, steps, how)
    st, want, _ = O.run(wl, O.F32, steps)
    assert np.array_equal(raster, want), f"first differing step {np.nonzero((raster != want).any(1))[0][:1]}"
    assert np.array_equal(np.asarray(v, np.float64), st.v)
    assert np.array_equal(np.asarray(r), st.r)
    # events: spikes times out-degree; a dense context counts every matrix
    # entry of a spiking row (zero weights included)
    deg = np.full(n, n) if how == "dense" else np.bincount(wl["pre"], minlength=n)
    assert ev == int((want.astype(np.int64) * deg).sum())
    assert want[-1].sum() > 0


_BIG = {}


@pytest.mark.parametrize("how", ["dense", "push", "pull"])
@pytest.mark.parametrize("p", [0.25, 1.0])
def test_paper_grid_n10000_exact(p, how):
    """The largest networks of Table 2 (N = 10,000: 25M and 100M synapses),
    which the benchmark times beside the paper's numbers: 12 steps (two input
    rounds; from step 2 on every neuron fires every step), bit for bit."""
    n, steps = 10_000, 12
    if p not in _BIG:
        wl = W.paper_grid(n, p, steps=steps)
        st, want, _ = O.run(wl, O.F32, steps)
        _BIG[p] = (wl, st, want)
    wl, st, want = _BIG[p]
    raster, v, r, ev = run(wl, steps, how)
    assert np.array_equal(raster, want), f"first differing step {np.nonzero((raster != want).any(1))[0][:1]}"
    assert np.array_equal(np.asarray(v, np.float64), st.v)
    assert np.array_equal(np.asarray(r), st.r)
    deg = np.full(n, n) if how == "dense" else np.bincount(wl["pre"], minlength=n)
    assert ev == int((want.astype(np.int64) * deg).sum())
    assert want[-1].sum() == n
