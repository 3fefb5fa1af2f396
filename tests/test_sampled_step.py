"""The sampled teacher-forced step (oracle/compare.py), used to check dense
networks too large for a host copy of their weights, must reproduce the full
oracle step exactly on every sampled neuron."""

import numpy as np
import pytest

from oracle import compare, oracle as O
from paper_2305_02510_gb300 import workloads as W


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sampled_step_equals_full_step(seed):
    rng = np.random.default_rng(seed)
    n, t = 300, 17
    wl = W.large_dense(n=n, steps=t + 1)
    # explicit events at step t (two on one neuron: summed in order) and
    # elsewhere, on top of the Poisson sources of every neuron
    wl["events"] = dict(step=np.array([t, t, t, t - 1], np.int32), neuron=np.array([5, 5, 40, 5], np.int32),
                        value=np.array([0.25, 0.5, 1.5, 9.0]))
    v = rng.normal(0.6, 0.3, n).astype(np.float32).astype(np.float64)
    r = rng.integers(0, 2, n).astype(np.int32)
    spk = (rng.random(n) < 0.2).astype(np.uint8)
    st = O.state_from(wl, t, v, r, spk[None, :])
    st, want, _ = O.run(wl, O.F32, 1, state=st)
    J = np.sort(rng.choice(n, 64, replace=False))
    J[0] = 5
    J = np.unique(np.concatenate([J, [40]]))
    spikers = np.nonzero(spk)[0]
    wcols = np.asarray(wl["dense_w"], np.float64)[spikers][:, J]
    row, sv, sr, _ = compare.sampled_dense_step(wl, t, J, v[J], r[J], spikers, wcols)
    assert np.array_equal(row, want[0][J])
    assert np.array_equal(sv, st.v[J])
    assert np.array_equal(sr, st.r[J])
    # the float64 trajectory likewise
    s64 = O.state_from(wl, t, v, r, spk[None, :])
    s64, want64, _ = O.run(wl, O.F64, 1, state=s64)
    row64, sv64, sr64, _ = compare.sampled_dense_step(wl, t, J, v[J], r[J], spikers, wcols, mode=O.F64)
    assert np.array_equal(row64, want64[0][J])
    assert np.array_equal(sv64, s64.v[J])
    assert np.array_equal(sr64, s64.r[J])
    assert compare.check_sampled_dense_step(wl, t, J, v[J], r[J], spikers, wcols, want64[0][J], s64.v[J],
                                            s64.r[J]) == int(want64[0][J].sum())


def test_sampled_step_catches_a_wrong_weight():
    rng = np.random.default_rng(9)
    n, t = 200, 4
    wl = W.large_dense(n=n, steps=t + 1)
    v = np.full(n, 0.95)
    r = np.zeros(n, np.int32)
    spk = (rng.random(n) < 0.3).astype(np.uint8)
    st = O.state_from(wl, t, v, r, spk[None, :])
    st, want, _ = O.run(wl, O.F32, 1, state=st)
    J = np.arange(0, n, 7)
    spikers = np.nonzero(spk)[0]
    wcols = np.asarray(wl["dense_w"], np.float64)[spikers][:, J].copy()
    wcols[3, 2] += 0.01
    with pytest.raises(compare.Divergence):
        compare.check_sampled_dense_step(wl, t, J, v[J], r[J], spikers, wcols, want[0][J], st.v[J], st.r[J])
