"""Dense networks beyond a host copy of their weights: the weights are drawn
on the device (workloads.huge_dense, up to the paper's 100,000-neuron
all-to-all network: 40 GB) and installed with sn_set_weights.  The executor
then uses column slabs of 64, 128 or 256 columns per block.  Checked by
sampled teacher-forced steps (oracle/compare.py: the oracle's own step of a
sub-network holding the sampled neurons and every neuron that spiked)."""

import numpy as np
import pytest

from oracle import compare
from paper_2305_02510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def sample(n, rng, k=384):
    """Random neurons plus each end of a few column slabs and the last neuron."""
    ends = [0, 31, 32, 63, 64, 127, 128, 255, 256, n - 1, n - 2, (n // 256) * 256, (n // 256) * 256 - 1]
    J = np.concatenate([rng.choice(n, k, replace=False), np.array(ends)])
    return np.unique(J[(J >= 0) & (J < n)])


@pytest.mark.parametrize("n", [20000, 20002, 40000, 40002, 60002, 100000])
def test_huge_dense_sampled_teacher_forced(n):
    """Column slabs of 64 (20,000), 128 (40,000) and 256 (60,002, 100,000)
    columns; n % 4 != 0 takes the scalar gather."""
    from paper_2305_02510_gb300 import sn as S
    wl = W.huge_dense(n=n, steps=64)
    w = W.dense_weights_on_device(wl, torch)
    ctx = S.from_workload(wl, record_steps=64, w_device=w)
    rng = np.random.default_rng(n)
    J = sample(n, rng)
    Jt = torch.tensor(J, device="cuda")
    checked, done, spikes = 0, 0, 0
    for t in (1, 2, 25):
        S.sn_run(ctx, t - done)
        v0, r0 = S.sn_get_state(ctx)
        prev = S.unpack_raster(S.sn_get_spikes(ctx, t - 1, t), n)[0]
        S.sn_run(ctx, 1)
        v1, r1 = S.sn_get_state(ctx)
        row = S.unpack_raster(S.sn_get_spikes(ctx, t, t + 1), n)[0]
        spikers = np.nonzero(prev)[0]
        Kt = torch.tensor(spikers, device="cuda", dtype=torch.int64)
        wcols = w.index_select(0, Kt).index_select(1, Jt).cpu().numpy()
        checked += compare.check_sampled_dense_step(wl, t, J, v0[J], r0[J], spikers, wcols, row[J], v1[J], r1[J])
        spikes += int(spikers.size)
        done = t + 1
    assert spikes > 100 and checked > 0
    steps, total, events = S.sn_get_counters(ctx)
    assert steps == done and events == total * n
    del ctx, w
    torch.cuda.empty_cache()


def test_set_weights_round_trip():
    """sn_set_weights installs exactly what sn_get_weights returns (dense:
    host and device arrays; sparse: input order)."""
    from paper_2305_02510_gb300 import sn as S
    wl = W.large_dense(n=257, steps=4)
    ctx = S.from_workload(wl)
    w2 = np.random.default_rng(0).normal(0, 0.05, 257 * 257).astype(np.float32)
    S.sn_set_weights(ctx, w2)
    assert np.array_equal(S.sn_get_weights(ctx), w2)
    wd = torch.tensor(w2[::-1].copy(), device="cuda")
    S.sn_set_weights(ctx, wd)
    assert np.array_equal(S.sn_get_weights(ctx), w2[::-1])
    ws = W.random_small(3, n=50, integer=False, steps=20, max_delay=3)
    c2 = S.from_workload(ws)
    new = np.random.default_rng(1).normal(0, 1, len(ws["pre"])).astype(np.float32)
    S.sn_set_weights(c2, new)
    assert np.array_equal(S.sn_get_weights(c2), new)


@pytest.mark.parametrize("prop", ["push", "pull"])
def test_set_weights_then_run(prop):
    """A sparse run after sn_set_weights (mid-run, after 30 steps) equals the
    oracle's run of the network with those weights from that step on."""
    from oracle import oracle as O
    from paper_2305_02510_gb300 import sn as S
    # integer-valued weights and parameters in a float network: every sum is
    # exact in both propagation modes, so the comparison is bit for bit
    ws = W.random_small(11, n=80, integer=True, steps=80, max_delay=4, p=0.15, events_rate=1.0)
    ws["dtype"] = "f32"
    c = S.from_workload(ws, record_steps=80)
    S.sn_set_propagation(c, S.SN_PULL if prop == "pull" else S.SN_PUSH)
    S.sn_run(c, 30)
    new = np.random.default_rng(2).integers(-3, 6, len(ws["pre"])).astype(np.float32)
    S.sn_set_weights(c, new)
    S.sn_run(c, 50)
    got = S.unpack_raster(S.sn_get_spikes(c, 0, 80), ws["n"])
    v, r = S.sn_get_state(c)
    st, want1, _ = O.run(ws, O.F32, 30)
    w2 = dict(ws, weight=new.astype(np.float64))
    st.w = np.asarray(new, np.float64).copy()
    st, want2, _ = O.run(w2, O.F32, 50, state=st)
    want = np.concatenate([want1, want2])
    first = np.nonzero((got != want).any(axis=1))[0]
    assert first.size == 0, f"first differing step {int(first[0])}"
    assert np.array_equal(np.asarray(v, np.float64), st.v)
    assert np.array_equal(np.asarray(r), st.r)
    assert want2.sum() > 0


def test_dense_weights_change_only_at_step_zero():
    from paper_2305_02510_gb300 import sn as S
    wl = W.large_dense(n=64, steps=4)
    ctx = S.from_workload(wl)
    S.sn_run(ctx, 2)
    with pytest.raises(S.SnError) as e:
        S.sn_set_weights(ctx, np.zeros(64 * 64, np.float32))
    assert e.value.status == S.SN_ESTATE
    S.sn_reset(ctx)
    S.sn_set_weights(ctx, np.zeros(64 * 64, np.float32))


def test_ff_engine_choice():
    from paper_2305_02510_gb300 import sn as S
    task = W.bptt_task(batch=3, sizes=(20, 10), steps=5, seed=1)
    from paper_2305_02510_gb300 import bptt
    net = bptt.FFNet.from_task(task)
    with pytest.raises(S.SnError) as e:             # batch 3: not a multiple of 8
        S.sn_ff_set_engine(net.ctx, S.SN_FF_TENSOR)
    assert e.value.status == S.SN_EUNSUPPORTED
    with pytest.raises(S.SnError) as e:
        S.sn_ff_set_engine(net.ctx, 7)
    assert e.value.status == S.SN_EINVAL
    S.sn_ff_set_engine(net.ctx, S.SN_FF_SIMT)
