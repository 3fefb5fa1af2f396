"""One shared dense integer network driven by many input trains, propagated
as an exact FP8 tensor-core GEMM (tcgen05): bit-exact against the oracle per
train, and bit-identical to the plain single-network dense path."""

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


def run(wl, steps, record=None):
    s = S()
    ctx = s.from_shared_workload(wl, record_steps=record or steps)
    s.sn_run(ctx, steps)
    s.sn_sync(ctx)
    bits = s.sn_get_spikes(ctx, 0, steps)
    v, r = s.sn_get_state(ctx)
    n, B = wl["n"], wl["batch"]
    return ctx, bits, v.reshape(B, n), r.reshape(B, n)


def train_raster(bits, n, b):
    w = n // 32
    return S().unpack_raster(np.ascontiguousarray(bits[:, b * w:(b + 1) * w]), n)


@pytest.mark.parametrize("n,B,T,trains", [(256, 128, 60, range(128)), (384, 256, 40, range(0, 256, 9)),
                                           (1024, 128, 30, range(0, 128, 17)),
                                           # 160 tiles of 128 x 128: more tiles than blocks, so the
                                           # state goes through global memory between steps
                                           (2048, 1280, 20, range(0, 1280, 97))])
def test_shared_bit_exact(n, B, T, trains):
    wl = W.shared_dense_i8(n=n, batch=B, steps=T)
    _, bits, v, r = run(wl, T)
    total = 0
    for b in trains:
        got = train_raster(bits, n, b)
        compare.check_int_run(wl, got, v[b], r[b], T, net_index=b)
        total += int(got.sum())
    assert total > 0


def test_shared_equals_plain_dense_path():
    """Integer weights and parameters held in float are exact, so the plain
    single-network dense path reproduces every train bit for bit."""
    s = S()
    wl = W.shared_dense_i8(n=256, batch=128, steps=50)
    _, bits, v, r = run(wl, 50)
    po = wl["poisson"]
    for b in (0, 5, 127):
        ctx = s.sn_create_dense(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"],
                                wl["dense_w_i8"].astype(np.float32), 1, record_steps=50)
        s.sn_set_poisson_stream(ctx, po["neuron"], po["rate"], po["amplitude"], po["seed"], b)
        s.sn_run(ctx, 50)
        got = s.unpack_raster(s.sn_get_spikes(ctx, 0, 50), wl["n"])
        vv, rr = s.sn_get_state(ctx)
        assert np.array_equal(got, train_raster(bits, wl["n"], b))
        assert np.array_equal(vv.astype(np.int64), v[b].astype(np.int64)) and np.array_equal(rr, r[b])


def test_shared_checkpoint_resume_bit_exact():
    """run(T) equals run(T1); save; load into a fresh context; run(T - T1):
    every train's spikes, the state and the counters."""
    s = S()
    T, T1 = 60, 23
    wl = W.shared_dense_i8(n=384, batch=256, steps=T)
    ctx, _, v_want, r_want = run(wl, T)
    want = s.sn_get_spikes(ctx, 0, T)
    a = s.from_shared_workload(wl, record_steps=T)
    s.sn_run(a, T1)
    first = s.sn_get_spikes(a, 0, T1)
    blob = s.sn_save(a)
    b = s.from_shared_workload(wl, record_steps=T)
    s.sn_load(b, blob)
    s.sn_run(b, T - T1)
    second = s.sn_get_spikes(b, T1, T)
    v, r = s.sn_get_state(b)
    assert np.array_equal(np.concatenate([first, second]), want)
    assert np.array_equal(v.reshape(v_want.shape), v_want) and np.array_equal(r.reshape(r_want.shape), r_want)
    assert tuple(s.sn_get_counters(b)) == tuple(s.sn_get_counters(ctx))
    # a checkpoint with another number of trains is refused
    other = s.from_shared_workload(W.shared_dense_i8(n=384, batch=128, steps=T), record_steps=T)
    with pytest.raises(s.SnError):
        s.sn_load(other, blob)


def test_shared_full_size_sampled():
    """8192 neurons x 256 trains, 500 steps: two trains bit-exact over the
    first 12 steps, then teacher-forced single steps of sampled trains."""
    s = S()
    wl = W.shared_dense_i8()
    n, B = wl["n"], wl["batch"]
    ctx = s.from_shared_workload(wl, record_steps=500)
    s.sn_run(ctx, 12)
    s.sn_sync(ctx)
    bits = s.sn_get_spikes(ctx, 0, 12)
    v, r = s.sn_get_state(ctx)
    v, r = v.reshape(B, n), r.reshape(B, n)
    for b in (0, 255):
        compare.check_int_run(wl, train_raster(bits, n, b), v[b], r[b], 12, net_index=b)
    for t in (200, 499):
        s.sn_run(ctx, t - s.sn_get_counters(ctx)[0])
        v0, r0 = s.sn_get_state(ctx)
        prev = s.sn_get_spikes(ctx, t - 1, t)
        s.sn_run(ctx, 1)
        v1, r1 = s.sn_get_state(ctx)
        row = s.sn_get_spikes(ctx, t, t + 1)
        for b in (3, 130):
            hist = train_raster(prev, n, b)
            st = O.state_from(wl, t, v0.reshape(B, n)[b], r0.reshape(B, n)[b], hist)
            st, want, _ = O.run(wl, O.INT, 1, state=st, net_index=b)
            assert np.array_equal(train_raster(row, n, b)[0], want[0]), (t, b)
            assert np.array_equal(v1.reshape(B, n)[b].astype(np.float64), st.v) and \
                np.array_equal(r1.reshape(B, n)[b], st.r)
    assert s.sn_get_counters(ctx)[1] > 0
