"""Comparison rules between a simulator run and the oracle.

TEST INFRASTRUCTURE ONLY (used by tests/, the smoke check and the benchmark's
parity probe).  Inputs are plain arrays; nothing here touches the GPU path.

Integer networks: rasters and states must be identical.
Float networks:   spikes identical except at neurons whose oracle state at the
                  threshold test lies within NEAR * |theta| of theta; states
                  within RTOL * max(|V|, |theta|) of the float32 mirror.  After
                  the first divergence the trajectories are chaotic, so later
                  steps are checked one at a time from the simulator's own
                  state (teacher forcing).
"""

from __future__ import annotations

import numpy as np

from . import oracle as O

RTOL = 1e-5
NEAR = 1e-4


class Divergence(AssertionError):
    pass


def _theta(wl):
    return np.asarray(np.asarray(wl["threshold"], np.float32), np.float64)


def check_int_run(wl, raster, v, r, steps, state=None, **run_kw):
    """Whole-run equality for integer networks.  Returns the oracle state.
    run_kw (net_index, poisson_seed) go to oracle.run."""
    st, want, _ = O.run(wl, O.INT, steps, state=state, **run_kw)
    bad = np.nonzero((raster != want).any(axis=1))[0]
    if bad.size:
        t = int(bad[0])
        j = np.nonzero(raster[t] != want[t])[0][:8]
        raise Divergence(f"integer raster differs first at step {st.t - steps + t}, neurons {j.tolist()}")
    if not np.array_equal(np.asarray(v, np.float64), st.v):
        j = np.nonzero(np.asarray(v, np.float64) != st.v)[0][:8]
        raise Divergence(f"integer state differs at neurons {j.tolist()}")
    if not np.array_equal(np.asarray(r), st.r):
        raise Divergence("refractory countdowns differ")
    return st


def check_float_run(wl, raster, v, r, steps, **run_kw):
    """Whole-run comparison for float networks.  Returns (first divergence
    step or None, oracle float32 state).  Raises on a violation."""
    st, want, _ = O.run(wl, O.F32, steps, record_v=True, **run_kw)
    th = _theta(wl)
    bad = np.nonzero((raster != want).any(axis=1))[0]
    if bad.size == 0:
        vv = np.asarray(v, np.float64)
        tol = RTOL * np.maximum(np.abs(st.v), np.abs(th))
        if not np.all(np.abs(vv - st.v) <= tol):
            j = int(np.argmax(np.abs(vv - st.v) / tol))
            raise Divergence(f"state of neuron {j}: {vv[j]!r} vs oracle {st.v[j]!r}")
        if not np.array_equal(np.asarray(r), st.r):
            raise Divergence("refractory countdowns differ")
        return None, st
    t = int(bad[0])
    j = np.nonzero(raster[t] != want[t])[0]
    gap = np.abs(st.ctrace[t, j] - th[j])
    if not np.all(gap < NEAR * np.abs(th[j])):
        k = int(np.argmax(gap))
        raise Divergence(f"spike of neuron {int(j[k])} at step {t} differs with oracle state "
                         f"{st.ctrace[t, j[k]]!r} not near threshold {th[j[k]]!r}")
    return t, st


def teacher_forced_step(wl, t, v_prev, r_prev, hist_rows, row, v, r, mode,
                        trace_prev=None, w_prev=None, w=None, trace=None):
    """One oracle step t from the simulator's state after step t-1, compared
    with the simulator's step t.  hist_rows: spikes of steps t-D .. t-1 as
    uint8 [D, n].  Returns the number of spikes compared."""
    st = O.state_from(wl, t, v_prev, r_prev, hist_rows, trace=trace_prev, w=w_prev)
    st, want, _ = O.run(wl, mode, 1, state=st, record_v=True)
    th = _theta(wl)
    if mode == O.INT:
        assert np.array_equal(row, want[0]), f"step {t}: integer spikes differ"
        assert np.array_equal(np.asarray(v, np.float64), st.v), f"step {t}: integer state differs"
        assert np.array_equal(np.asarray(r), st.r)
        return int(want[0].sum())
    diff = np.nonzero(row != want[0])[0]
    if diff.size:
        gap = np.abs(st.ctrace[0, diff] - th[diff])
        if not np.all(gap < NEAR * np.abs(th[diff])):
            k = int(np.argmax(gap))
            raise Divergence(f"teacher-forced step {t}: neuron {int(diff[k])} spike differs, oracle "
                             f"state {st.ctrace[0, diff[k]]!r} vs threshold {th[diff[k]]!r}")
    same = np.ones(row.shape, bool)
    same[diff] = False
    vv = np.asarray(v, np.float64)
    tol = RTOL * np.maximum(np.abs(st.v), np.abs(th))
    ok = (np.abs(vv - st.v) <= tol) | ~same
    if not np.all(ok):
        j = int(np.nonzero(~ok)[0][0])
        raise Divergence(f"teacher-forced step {t}: state of neuron {j}: {vv[j]!r} vs {st.v[j]!r}")
    assert np.array_equal(np.asarray(r)[same], st.r[same])
    if w is not None:
        # weights changed by STDP: identical where both sides saw the same spikes
        ww = np.asarray(w, np.float64).reshape(-1)
        if diff.size == 0:
            assert np.array_equal(ww, st.w), f"step {t}: STDP weights differ"
    if trace is not None and diff.size == 0:
        assert np.array_equal(np.asarray(trace, np.float64), st.trace), f"step {t}: traces differ"
    return int(want[0].sum())


def sampled_dense_step(wl, t, J, v_prev, r_prev, spikers, wcols, mode=O.F32):
    """Oracle step t of a dense network with delay 1, for the neurons J only,
    from outside state (teacher forcing on a sample, for networks whose full
    weight matrix is too large for the host).

    J: ascending neuron indices; v_prev, r_prev: their state after step t-1;
    spikers: ascending indices of the neurons that spiked at t-1; wcols:
    [len(spikers), len(J)] = W[spikers][:, J].  The oracle runs one step of a
    sub-network: len(spikers) source neurons that spiked at t-1 (indices in
    the same ascending order, so the synaptic sum keeps the full network's
    order) and the neurons J with their parameters, joined by the synapses of
    wcols; J's Poisson draws of step t (the full network's stream, index j)
    become explicit events after J's own events of step t.  Returns (spikes,
    v, r, compared state), each of length len(J)."""
    J = np.asarray(J, np.int64)
    K = int(len(spikers))
    nq = int(J.size)
    n2 = K + nq
    f = O.canon(wl, mode)
    sub = dict(n=n2, dtype=wl["dtype"], max_delay=1, steps=1, stdp=None)
    big = np.full(K, 1e30)
    sub["threshold"] = np.concatenate([big, f(wl["threshold"])[J]])
    sub["leak"] = np.concatenate([np.zeros(K), f(wl["leak"])[J]])
    sub["reset"] = np.concatenate([np.zeros(K), f(wl["reset"])[J]])
    sub["refractory"] = np.concatenate([np.zeros(K, np.int32), np.asarray(wl["refractory"], np.int32)[J]])
    pre = np.repeat(np.arange(K, dtype=np.int32), nq)
    post = np.tile(np.arange(K, n2, dtype=np.int32), K)
    sub.update(pre=pre, post=post, weight=np.asarray(wcols, np.float64).reshape(-1),
               delay=np.ones(pre.size, np.int32))
    # J's external input of step t: its explicit events in order, then its
    # Poisson amplitude if the full network's source fires
    ev = wl["events"]
    pos = {int(j): K + q for q, j in enumerate(J)}
    es, en, evv = [], [], []
    for s_, j_, v_ in zip(np.asarray(ev["step"]), np.asarray(ev["neuron"]), np.asarray(ev["value"])):
        if int(s_) == t and int(j_) in pos:
            es.append(t), en.append(pos[int(j_)]), evv.append(float(v_))
    po = wl["poisson"]
    thr = O.rate_to_u32(np.asarray(po["rate"], np.float32).astype(np.float64))
    for k, j in enumerate(np.asarray(po["neuron"])):
        if int(j) in pos and O.poisson_u32(int(po["seed"]), 0, int(t), int(j)) < thr[k]:
            es.append(t), en.append(pos[int(j)]), evv.append(float(po["amplitude"][k]))
    sub["events"] = dict(step=np.asarray(es, np.int32), neuron=np.asarray(en, np.int32),
                         value=np.asarray(evv, np.float64))
    sub["poisson"] = dict(neuron=np.zeros(0, np.int32), rate=np.zeros(0), amplitude=np.zeros(0), seed=0)
    v0 = np.concatenate([np.zeros(K), np.asarray(v_prev, np.float64)])
    r0 = np.concatenate([np.zeros(K, np.int32), np.asarray(r_prev, np.int32)])
    hist = np.zeros((1, n2), np.uint8)
    hist[0, :K] = 1
    st = O.state_from(sub, t, v0, r0, hist)
    st, raster, _ = O.run(sub, mode, 1, state=st, record_v=True)
    return raster[0, K:], st.v[K:], st.r[K:], st.ctrace[0, K:]


def check_sampled_dense_step(wl, t, J, v_prev, r_prev, spikers, wcols, row, v, r):
    """Compare the simulator's step t on the sample J (spikes `row`, state v,
    r, each of length len(J)) with the float64 oracle's sampled step: spikes
    equal except where the oracle's compared state is within NEAR * |theta|
    of theta; state within RTOL * max(|V|, |theta|) of the oracle's.  These
    networks sum thousands of weights per step, and the float32 mirror's
    sequential sum then drifts from the exact one by up to ~1e-5 itself, so
    the float64 potentials are the reference here.  Returns the number of
    spikes compared."""
    want, wv, wr, ct = sampled_dense_step(wl, t, J, v_prev, r_prev, spikers, wcols, mode=O.F64)
    th = _theta(wl)[np.asarray(J)]
    diff = np.nonzero(np.asarray(row) != want)[0]
    if diff.size and not np.all(np.abs(ct[diff] - th[diff]) < NEAR * np.abs(th[diff])):
        k = int(diff[np.argmax(np.abs(ct[diff] - th[diff]))])
        raise Divergence(f"sampled step {t}: neuron {int(J[k])} spike differs, oracle state {ct[k]!r}")
    same = np.ones(len(J), bool)
    same[diff] = False
    vv = np.asarray(v, np.float64)
    ok = (np.abs(vv - wv) <= RTOL * np.maximum(np.abs(wv), np.abs(th))) | ~same
    if not np.all(ok):
        k = int(np.nonzero(~ok)[0][0])
        raise Divergence(f"sampled step {t}: state of neuron {int(J[k])}: {vv[k]!r} vs {wv[k]!r}")
    assert np.array_equal(np.asarray(r)[same], wr[same])
    return int(want.sum())
