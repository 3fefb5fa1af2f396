"""Pins for the CPU oracle: facts fixed by the paper's rules and by
mathematics, independent of the oracle's own code.

  * closed-form firing period of one LIF neuron under constant input
  * spike arrival along delay chains = sum of the delays (Section 2.1 proxies,
    Section 2.2 delay registers)
  * no spike inside a refractory period (Section 2.1)
  * the matrix formulation with proxy neurons (Section 2.1) and the literal
    per-synapse shift-register formulation (Section 2.2) give identical rasters
  * linear superposition of delivered weights against a float64 matrix product
  * exhaustive brute force on 2-neuron networks
  * hand-computed pair-based STDP updates and clipping
  * the published SplitMix64 test vector and the Poisson source rate
  * the all-to-all matrix form equals the per-synapse form of the same
    network (integer and float, with and without STDP)
  * a state rebuilt from outside values continues like the uninterrupted run
"""

import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle.formulations import abm_registers, mat_proxy
from paper_2305_02510_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = [O.F64, O.F32, O.INT]


def single_neuron(theta, leak, reset, refr, inp, steps, dtype):
    wl = W._base(1, dtype, theta, leak, reset, refr, 1, steps)
    wl.update(pre=np.zeros(0, np.int32), post=np.zeros(0, np.int32),
              weight=np.zeros(0), delay=np.zeros(0, np.int32))
    wl["events"] = dict(step=np.arange(steps, dtype=np.int32),
                        neuron=np.zeros(steps, np.int32), value=np.full(steps, float(inp)))
    return wl


def closed_form_spikes(theta, leak, reset, refr, inp, steps):
    """Spike steps of one neuron started at rest under input `inp` per step.

    From rest V = reset: V_k = reset + I + (k-1)(I - leak) while I > leak, so
    the first crossing after a reset is k* = 1 if reset + I > theta, else
    floor((theta - reset - I)/(I - leak)) + 2.  With I <= leak the state stays
    at reset + I.  A spike at t blocks t+1..t+R and the state keeps rising
    meanwhile, so consecutive spikes are max(k*, R+1) apart."""
    if reset + inp > theta:
        k = 1
    elif inp <= leak:
        return []
    else:
        k = math.floor((theta - reset - inp) / (inp - leak)) + 2
    period = max(k, refr + 1)
    return list(range(k - 1, steps, period))


CASES = [
    # theta, leak, reset, R, I
    (1.0, 0.125, 0.0, 0, 0.25),
    (1.0, 0.125, 0.0, 3, 0.25),
    (1.0, 0.125, 0.0, 9, 0.25),
    (1.0, 0.25, 0.0, 0, 0.25),      # I == leak: never fires
    (0.5, 0.25, 0.0, 2, 0.75),      # I > theta: fires every R+1
    (1.0, 0.0, 0.0, 0, 0.5),
    (1.0, 0.0625, -0.5, 1, 0.375),  # negative reset
    (3.0, 0.5, 0.0, 0, 0.625),
]
INT_CASES = [(10, 1, 0, 1, 3), (10, 1, 0, 0, 11), (20, 1, -5, 4, 2), (7, 2, 0, 0, 2)]


@pytest.mark.parametrize("mode", [O.F64, O.F32])
@pytest.mark.parametrize("case", CASES)
def test_closed_form_period(case, mode):
    th, lk, rs, R, I = case
    steps = 200
    wl = single_neuron(th, lk, rs, R, I, steps, "f32")
    _, raster, _ = O.run(wl, mode, steps)
    got = list(np.nonzero(raster[:, 0])[0])
    assert got == closed_form_spikes(th, lk, rs, R, I, steps)


@pytest.mark.parametrize("case", INT_CASES)
def test_closed_form_period_int(case):
    th, lk, rs, R, I = case
    steps = 300
    wl = single_neuron(th, lk, rs, R, I, steps, "i32")
    _, raster, _ = O.run(wl, O.INT, steps)
    assert list(np.nonzero(raster[:, 0])[0]) == closed_form_spikes(th, lk, rs, R, I, steps)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("delays", [[1], [3, 1, 4, 2], [5, 5, 5], [2, 7, 1, 1, 6, 3]])
def test_delay_chain_arrival(delays, mode):
    m = len(delays)
    n = m + 1
    D = max(delays)
    dtype = "i32" if mode == O.INT else "f32"
    wl = W._base(n, dtype, 1, 1, 0, 0, D, 0)
    wl.update(pre=np.arange(m, dtype=np.int32), post=np.arange(1, n, dtype=np.int32),
              weight=np.full(m, 2.0), delay=np.array(delays, np.int32))
    t0 = 5
    wl["events"] = dict(step=np.array([t0], np.int32), neuron=np.array([0], np.int32),
                        value=np.array([2.0]))
    steps = t0 + sum(delays) + 10
    _, raster, _ = O.run(wl, mode, steps)
    for k in range(n):
        assert list(np.nonzero(raster[:, k])[0]) == [t0 + sum(delays[:k])]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("delays,axonal", [([1], [0]), ([3, 1, 4], [2, 0, 5]), ([1, 1, 1, 1], [3, 3, 0, 1])])
def test_axonal_delay_chain_arrival(delays, axonal, mode):
    """Section 2.2's axonal delay (a neuron parameter): along a chain, neuron k
    fires at t0 + sum over earlier hops of (axonal delay + synaptic delay).
    A fan-out neuron adds its axonal delay to every outgoing synapse."""
    m = len(delays)
    n = m + 3
    D = max(d + a for d, a in zip(delays, axonal)) + 2
    dtype = "i32" if mode == O.INT else "f32"
    wl = W._base(n, dtype, 1, 1, 0, 0, D, 0)
    ax = np.zeros(n, np.int32)
    ax[:m] = axonal
    ax[m] = 1                      # the end of the chain fans out to two neurons
    wl.update(pre=np.concatenate([np.arange(m), [m, m]]).astype(np.int32),
              post=np.concatenate([np.arange(1, n - 2), [m + 1, m + 2]]).astype(np.int32),
              weight=np.full(m + 2, 2.0), delay=np.array(list(delays) + [1, 2], np.int32), axonal_delay=ax)
    t0 = 5
    wl["events"] = dict(step=np.array([t0], np.int32), neuron=np.array([0], np.int32),
                        value=np.array([2.0]))
    hop = [d + a for d, a in zip(delays, axonal)]
    steps = t0 + sum(hop) + 10
    _, raster, _ = O.run(wl, mode, steps)
    for k in range(m + 1):
        assert list(np.nonzero(raster[:, k])[0]) == [t0 + sum(hop[:k])]
    tm = t0 + sum(hop)
    assert list(np.nonzero(raster[:, m + 1])[0]) == [tm + 1 + 1]
    assert list(np.nonzero(raster[:, m + 2])[0]) == [tm + 1 + 2]
    # all axonal delays 0: the plain network
    wl0 = dict(wl, axonal_delay=np.zeros(n, np.int32))
    wl1 = {k: v for k, v in wl.items() if k != "axonal_delay"}
    assert np.array_equal(O.run(wl0, mode, steps)[1], O.run(wl1, mode, steps)[1])


@pytest.mark.parametrize("seed", range(60))
def test_axonal_oracle_equals_shared_axon_proxies(seed):
    """The oracle composes each synapse's delay with its pre-neuron's axonal
    delay; the matrix formulation instead routes all of a neuron's outgoing
    synapses through one shared chain of axonal proxy neurons.  Rasters must
    agree bit for bit (integer networks)."""
    wl = W.random_small(7000 + seed, integer=True, steps=120, events_rate=0.5)
    rng = np.random.default_rng(seed)
    wl["axonal_delay"] = rng.integers(0, 4, wl["n"]).astype(np.int32)
    wl["max_delay"] = int(wl["max_delay"]) + 3
    _, want, _ = O.run(wl, O.INT, 120)
    got, _, _ = mat_proxy(wl, 120, integer=True)
    assert np.array_equal(got, want)
    assert want.sum() > 0 or len(wl["pre"]) == 0


def _check_isi(raster, refr):
    for j in range(raster.shape[1]):
        t = np.nonzero(raster[:, j])[0]
        if t.size > 1:
            assert np.diff(t).min() >= refr[j] + 1


@pytest.mark.parametrize("seed", range(10))
def test_refractory_invariant_random(seed):
    wl = W.random_small(seed, integer=bool(seed % 2), steps=300, events_rate=0.5)
    mode = O.INT if seed % 2 else O.F32
    _, raster, _ = O.run(wl, mode, 300)
    _check_isi(raster, wl["refractory"])


def test_refractory_invariant_tiny():
    for integer in (False, True):
        wl = W.tiny(integer=integer)
        _, raster, _ = O.run(wl, O.INT if integer else O.F32, 1000)
        assert raster.sum() > 0
        _check_isi(raster, wl["refractory"])


@pytest.mark.parametrize("block", range(4))
def test_mat_proxy_matches_oracle(block):
    """Integer mode: bit-identical rasters and final states on 50 random
    networks per block (N <= 20, D <= 4, T = 120)."""
    for seed in range(block * 50, block * 50 + 50):
        wl = W.random_small(1000 + seed, integer=True, steps=120, events_rate=0.6)
        st, raster, _ = O.run(wl, O.INT, 120)
        mraster, mv, mr = mat_proxy(wl, 120, integer=True)
        assert np.array_equal(raster, mraster), seed
        assert np.array_equal(st.v, mv.astype(np.float64)), seed
        assert np.array_equal(st.r, mr), seed


@pytest.mark.parametrize("seed", range(12))
def test_abm_registers_match_oracle(seed):
    wl = W.random_small(2000 + seed, integer=True, steps=80, events_rate=0.6)
    st, raster, _ = O.run(wl, O.INT, 80)
    araster, av, ar = abm_registers(wl, 80)
    assert np.array_equal(raster, araster)
    assert np.array_equal(st.v, av)
    assert np.array_equal(st.r, ar)


def test_mat_proxy_float_close():
    """Float64 oracle vs float64 matrix form on float nets: same rasters while
    no state sits within 1e-9 of its threshold."""
    for seed in range(20):
        wl = W.random_small(3000 + seed, integer=False, steps=60, events_rate=0.6)
        st, raster, _ = O.run(wl, O.F64, 60, record_v=True)
        mraster, _, _ = mat_proxy(wl, 60, integer=False)
        bad = np.nonzero((raster != mraster).any(axis=1))[0]
        if bad.size:
            t = bad[0]
            j = np.nonzero(raster[t] != mraster[t])[0]
            assert np.all(np.abs(st.ctrace[t, j] - wl["threshold"][j]) < 1e-9)


@pytest.mark.parametrize("mode", [O.F64, O.INT])
def test_linear_superposition(mode):
    """Receivers with an unreachable threshold and no leak accumulate every
    delivered weight: V_j(T) = sum_k w_k * #{t < T - d_k + 1 : pre_k spiked at t}."""
    rng = np.random.default_rng(7)
    nd, nr = 12, 9
    n = nd + nr
    m = 80
    pre = rng.integers(0, nd, m).astype(np.int32)
    post = rng.integers(nd, n, m).astype(np.int32)
    delay = rng.integers(1, 6, m).astype(np.int32)
    integer = mode == O.INT
    w = rng.integers(-4, 6, m).astype(np.float64) if integer else rng.normal(0, 1, m)
    th = np.concatenate([np.full(nd, 1.0), np.full(nr, 1e30 if not integer else 2.0**40)])
    wl = W._base(n, "i32" if integer else "f32", th, 0, 0, 0, 5, 0)
    wl["leak"][:nd] = 1.0
    wl.update(pre=pre, post=post, weight=w, delay=delay)
    T = 150
    ev_t = rng.integers(0, T, 300).astype(np.int32)
    ev_j = rng.integers(0, nd, 300).astype(np.int32)
    wl["events"] = dict(step=ev_t, neuron=ev_j, value=np.full(300, 2.0))
    st, raster, _ = O.run(wl, mode, T)
    wq = np.asarray(w, np.float32).astype(np.float64) if not integer else w
    # counts[k] = spikes of pre_k early enough to arrive by step T-1
    cum = np.cumsum(raster[:, :nd], axis=0)
    cnt = np.array([cum[T - 1 - delay[k], pre[k]] if T - 1 - delay[k] >= 0 else 0
                    for k in range(m)], np.float64)
    M = np.zeros((m, nr))
    M[np.arange(m), post - nd] = 1.0
    expect = (cnt * wq) @ M
    got = st.v[nd:]
    if integer:
        assert np.array_equal(got, expect)
    else:
        np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-12)
    assert raster[:, nd:].sum() == 0


def test_brute_force_two_neurons():
    """Every 2-neuron network with synapses 0->1 and/or 1->0, delays 1..3,
    weights in {-2, 1, 3}, refractory 0/1, leak 0/1: the C oracle and the
    literal shift-register formulation agree."""
    rng = np.random.default_rng(3)
    ev_t = rng.integers(0, 30, 12).astype(np.int32)
    ev_j = rng.integers(0, 2, 12).astype(np.int32)
    count = 0
    for links in ([(0, 1)], [(1, 0)], [(0, 1), (1, 0)], [(0, 1), (0, 1)]):
        for ds in np.ndindex(*(3,) * len(links)):
            for ws in np.ndindex(*(3,) * len(links)):
                for R in (0, 1):
                    for lk in (0, 1):
                        wl = W._base(2, "i32", 2, lk, 0, R, 3, 30)
                        wl.update(pre=np.array([a for a, _ in links], np.int32),
                                  post=np.array([b for _, b in links], np.int32),
                                  weight=np.array([(-2, 1, 3)[x] for x in ws], np.float64),
                                  delay=np.array([d + 1 for d in ds], np.int32))
                        wl["events"] = dict(step=ev_t, neuron=ev_j, value=np.full(12, 3.0))
                        _, raster, _ = O.run(wl, O.INT, 30)
                        araster, _, _ = abm_registers(wl, 30)
                        assert np.array_equal(raster, araster)
                        count += 1
    assert count > 300


def _stdp_pair(t_pre, t_post, w0, a_plus=0.01, a_minus=0.012, decay=0.9, steps=30):
    wl = W._base(2, "f32", 1.0, 10.0, 0.0, 0, 1, steps)
    wl.update(pre=np.array([0], np.int32), post=np.array([1], np.int32),
              weight=np.array([w0]), delay=np.array([1], np.int32))
    wl["events"] = dict(step=np.array([t_pre, t_post], np.int32),
                        neuron=np.array([0, 1], np.int32), value=np.array([2.0, 2.0]))
    wl["stdp"] = dict(decay=decay, a_plus=a_plus, a_minus=a_minus, wmin=-1.0, wmax=1.0)
    st, raster, _ = O.run(wl, O.F64, steps)
    assert raster[t_pre, 0] == 1 and raster[t_post, 1] == 1
    return st


@pytest.mark.parametrize("dt", [1, 2, 5])
def test_stdp_pre_before_post(dt):
    st = _stdp_pair(3, 3 + dt, 0.0)
    assert st.w[0] == pytest.approx(0.01 * 0.9 ** (dt - 1), rel=1e-12)


@pytest.mark.parametrize("dt", [1, 3, 6])
def test_stdp_post_before_pre(dt):
    st = _stdp_pair(3 + dt, 3, 0.0)
    assert st.w[0] == pytest.approx(-0.012 * 0.9 ** (dt - 1), rel=1e-12)


def test_stdp_simultaneous_and_clip():
    assert _stdp_pair(4, 4, 0.0).w[0] == 0.0          # both traces still 0
    assert _stdp_pair(3, 4, 0.995).w[0] == 1.0        # 0.995 + 0.01 clipped
    assert _stdp_pair(4, 3, -0.995).w[0] == -1.0      # -0.995 - 0.012 clipped


def test_stdp_trace_decay():
    st = _stdp_pair(2, 9, 0.0, steps=15)
    # trace of neuron 0 after its spike at 2, read after step 14: 0.9^12
    assert st.trace[0] == pytest.approx(0.9 ** 12, rel=1e-12)
    assert st.trace[1] == pytest.approx(0.9 ** 5, rel=1e-12)


def test_event_sum_order_fp32():
    """Explicit events of one (t, j) add in the order given, in float32 when
    mirroring float: (1e8 + 1) - 1e8 = 0 in float32 but 1 in float64."""
    wl = W._base(1, "f32", 1e30, 0.0, 0.0, 0, 1, 1)
    wl.update(pre=np.zeros(0, np.int32), post=np.zeros(0, np.int32),
              weight=np.zeros(0), delay=np.zeros(0, np.int32))
    wl["events"] = dict(step=np.zeros(3, np.int32), neuron=np.zeros(3, np.int32),
                        value=np.array([1e8, 1.0, -1e8]))
    assert O.run(wl, O.F32, 1)[0].v[0] == 0.0
    assert O.run(wl, O.F64, 1)[0].v[0] == 1.0


def test_splitmix64_published_vector():
    vals = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    g = 0x9E3779B97F4A7C15
    assert [O.splitmix64((1234567 + k * g) % 2**64) for k in range(5)] == vals


def test_poisson_rate_and_streams():
    L = O.lib()
    thr = int(O.rate_to_u32(0.05))
    n = 0
    hits = 0
    for t in range(200):
        for j in range(500):
            hits += L.orc_poisson_u32(99, 3, t, j) < thr
            n += 1
    p = hits / n
    assert abs(p - 0.05) < 5 * math.sqrt(0.05 * 0.95 / n)
    a = [L.orc_poisson_u32(99, 3, 7, j) for j in range(64)]
    b = [L.orc_poisson_u32(99, 4, 7, j) for j in range(64)]
    c = [L.orc_poisson_u32(99, 3, 8, j) for j in range(64)]
    assert a != b and a != c
    assert O.rate_to_u32(1.0) == 2**32 - 1 and O.rate_to_u32(0.0) == 0


def test_resume_equals_single_run():
    """Running T steps equals running T1 then T - T1 from the saved state."""
    wl = W.tiny(integer=False)
    st, r_all, _ = O.run(wl, O.F32, 400)
    st1, r1, _ = O.run(wl, O.F32, 150)
    st2, r2, _ = O.run(wl, O.F32, 250, state=st1)
    assert np.array_equal(r_all, np.concatenate([r1, r2]))
    assert np.array_equal(st.v, st2.v)


def test_fp32_mirror_tracks_fp64():
    """The float32 mirror stays within 1e-5 (relative to max(|V|, theta)) of
    the float64 trajectory until the first step where they spike differently,
    and that step has a state within 1e-4 * theta of its threshold."""
    wl = W.tiny(integer=False)
    s64, r64, v64 = O.run(wl, O.F64, 1000, record_v=True)
    _, r32, v32 = O.run(wl, O.F32, 1000, record_v=True)
    diff = np.nonzero((r64 != r32).any(axis=1))[0]
    end = diff[0] if diff.size else 1000
    th = np.asarray(wl["threshold"])
    scale = np.maximum(np.abs(v64[:end]), th)
    assert np.all(np.abs(v32[:end] - v64[:end]) <= 1e-5 * scale)
    if diff.size:
        t = diff[0]
        j = np.nonzero(r64[t] != r32[t])[0]
        assert np.all(np.abs(s64.ctrace[t, j] - th[j]) < 1e-4 * th[j])


def dense_as_synapses(wl, diagonal=True):
    """The same network in the per-synapse form: one synapse i -> j of the
    matrix's delay for every entry W[i][j] (row = pre, Section 2.1), listed in
    row-major order; without the diagonal when it is left out."""
    n = wl["n"]
    w = np.asarray(wl["dense_w"] if "dense_w" in wl else wl["dense_w_i8"], np.float64)
    mask = np.ones((n, n), bool) if diagonal else ~np.eye(n, dtype=bool)
    i, j = np.nonzero(mask)
    d = int(wl["dense_delay"])
    out = {k: v for k, v in wl.items() if k not in ("dense_w", "dense_w_i8", "dense_delay")}
    out.update(pre=i.astype(np.int32), post=j.astype(np.int32), weight=w[i, j],
               delay=np.full(i.size, d, np.int32), max_delay=max(int(wl["max_delay"]), d))
    return out, mask


@pytest.mark.parametrize("delay", [1, 3])
def test_dense_form_equals_synapse_form_int(delay):
    """The oracle's matrix form (the previous spike vector times W, row =
    pre, diagonal included) gives the same integer run as the per-synapse
    form of the same network: a transposed matrix, a dropped diagonal or a
    wrong delay in the matrix form fails this."""
    n, T = 48, 80
    wl = W.shared_dense_i8(n=n, batch=1, steps=T)       # theta 40, Poisson amplitude 41
    rng = np.random.default_rng(11 + delay)
    w = rng.integers(-8, 9, size=(n, n)).astype(np.int8)
    w[np.triu_indices(n, 1)] = np.abs(w[np.triu_indices(n, 1)])   # asymmetric
    wl.update(dense_w_i8=w, dense_delay=delay, max_delay=delay)
    a, ra, _ = O.run(wl, O.INT, T)
    syn, _ = dense_as_synapses(wl)
    b, rb, _ = O.run(syn, O.INT, T)
    assert ra.sum() > 0
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.r, b.r)
    # the transposed matrix is a different network
    wt = dict(wl, dense_w_i8=np.ascontiguousarray(w.T))
    _, rt, _ = O.run(wt, O.INT, T)
    assert not np.array_equal(rt, ra)


@pytest.mark.parametrize("mode", [O.F32, O.F64])
@pytest.mark.parametrize("stdp", [False, True])
def test_dense_form_equals_synapse_form_float(mode, stdp):
    """Float runs of the matrix form and the per-synapse form are identical
    bit for bit (both add a post-neuron's inputs in ascending pre order), and
    with STDP so are the weights after the run (the matrix form's rule skips
    the diagonal, which is not a synapse)."""
    n, T = 64, 60
    wl = W.large_dense(n=n, stdp=stdp, steps=T)
    wl["dense_w"] = (wl["dense_w"] * np.float32(10.0)).astype(np.float32)   # N(0, 0.2), W_ii = 0
    a, ra, _ = O.run(wl, mode, T)
    syn, mask = dense_as_synapses(wl, diagonal=False)
    b, rb, _ = O.run(syn, mode, T)
    assert ra.sum() > 0
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.r, b.r)
    if stdp:
        wa = a.w.reshape(n, n)
        assert np.array_equal(wa[mask], b.w)
        assert np.all(np.diag(wa) == 0)
        assert not np.array_equal(wa, np.asarray(wl["dense_w"], np.float64))   # plasticity acted


@pytest.mark.parametrize("kind", ["sparse", "dense-stdp"])
def test_state_from_rebuilds_the_run(kind):
    """A state rebuilt from V, the refractory countdowns, the last D spike
    rows (oldest first), the traces and the weights continues exactly like
    the uninterrupted run: the teacher-forced comparisons rest on this."""
    if kind == "sparse":
        wl = W.tiny(integer=False, steps=200)          # delays 1..4
    else:
        wl = W.large_dense(n=64, stdp=True, steps=200)
        wl["dense_w"] = (wl["dense_w"] * np.float32(10.0)).astype(np.float32)
    D, t, k = wl["max_delay"], 120, 60
    full, raster, _ = O.run(wl, O.F32, t + k)
    part, r1, _ = O.run(wl, O.F32, t)
    st = O.state_from(wl, t, part.v, part.r, raster[t - D:t], trace=part.trace, w=part.w)
    st2, r2, _ = O.run(wl, O.F32, k, state=st)
    assert raster[t:].sum() > 0
    assert np.array_equal(r2, raster[t:])
    assert np.array_equal(st2.v, full.v) and np.array_equal(st2.r, full.r)
    assert np.array_equal(st2.w, full.w)
    # the rows in the other order do not give the same continuation
    if raster[t - D:t].any() and not np.array_equal(raster[t - D:t], raster[t - D:t][::-1]):
        bad = O.state_from(wl, t, part.v, part.r, raster[t - D:t][::-1], trace=part.trace, w=part.w)
        _, rb, _ = O.run(wl, O.F32, k, state=bad)
        assert not np.array_equal(rb, raster[t:])


def test_integer_overflow_is_detected():
    """Integer mode: a state that leaves the int32 range is an error.  One
    neuron gets 2^23 - 1 every step with no leak: 256 steps reach
    2^31 - 256 (fine), the 257th passes 2^31."""
    n, T = 4, 300
    wl = W._base(n, "i32", 2.0 ** 31, 0, 0, 0, 1, T)
    wl.update(pre=np.zeros(0, np.int32), post=np.zeros(0, np.int32), weight=np.zeros(0),
              delay=np.zeros(0, np.int32))
    wl["events"] = dict(step=np.arange(T, dtype=np.int32), neuron=np.zeros(T, np.int32),
                        value=np.full(T, 2.0 ** 23 - 1))
    st, raster, _ = O.run(wl, O.INT, 256)
    assert st.v[0] == 256 * (2 ** 23 - 1) and raster.sum() == 0
    with pytest.raises(RuntimeError):
        O.run(wl, O.INT, 257)


@pytest.mark.parametrize("kind", ["sparse-float", "sparse-int", "dense-stdp"])
def test_threads_do_not_change_results(kind):
    """The per-neuron loop on several threads (the CPU baseline's
    multi-threaded timing) gives the single-threaded run bit for bit."""
    if kind == "sparse-float":
        wl = W.large_sparse(integer=False, n=3000, k=40, steps=60)
    elif kind == "sparse-int":
        wl = W.large_sparse(integer=True, n=3000, k=40, steps=60)
    else:
        wl = W.large_dense(n=300, stdp=True, steps=60)
    mode = O.INT if wl["dtype"] == "i32" else O.F32
    out = []
    for k in (1, 4):
        O.set_threads(k)
        try:
            st, raster, _ = O.run(wl, mode, 60, record_v=True)
        finally:
            O.set_threads(1)
        out.append((st, raster))
    (a, ra), (b, rb) = out
    assert ra.sum() > 0 and np.array_equal(ra, rb)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.r, b.r)
    assert np.array_equal(a.ctrace, b.ctrace) and np.array_equal(a.w, b.w)


def test_integer_overflow_is_detected_on_threads():
    """As above, with the growing neuron in the middle of a 64-neuron loop
    split over three threads: steps 0..255 stay in range, step 256 is an
    error."""
    n, T = 64, 300
    wl = W._base(n, "i32", 2.0 ** 31, 0, 0, 0, 1, T)
    wl.update(pre=np.zeros(0, np.int32), post=np.zeros(0, np.int32), weight=np.zeros(0),
              delay=np.zeros(0, np.int32))
    wl["events"] = dict(step=np.arange(T, dtype=np.int32), neuron=np.full(T, 37, np.int32),
                        value=np.full(T, 2.0 ** 23 - 1))
    O.set_threads(3)
    try:
        st, raster, _ = O.run(wl, O.INT, 256)
        assert st.v[37] == 256 * (2 ** 23 - 1) and raster.sum() == 0
        with pytest.raises(RuntimeError):
            O.run(wl, O.INT, 257)
    finally:
        O.set_threads(1)


def test_fp32_mirror_drifts_past_the_state_bound_over_long_dense_runs():
    """The reading behind the long-launch check of the 100,000-neuron dense
    network: over 200 free-running steps of a dense network with the same
    per-step input variance (thousands of weights summed per step), the
    float32 mirror's states, with every spike equal to float64's, drift from
    float64 by more than 1e-5 * max(|V|, theta) (about 2.6 times it at 4,000
    neurons).  The 1e-5 bound is a per-step rule (teacher-forced steps); a
    state at the end of a long free run is held to a multiple of what
    float32 itself reaches."""
    n, T = 4000, 200
    wl = W.large_dense(n=n, steps=T)
    wl["dense_w"] = (wl["dense_w"] * np.sqrt(16384.0 / n)).astype(np.float32)
    O.set_threads(4)
    try:
        a, ra, _ = O.run(wl, O.F64, T)
        b, rb, _ = O.run(wl, O.F32, T)
    finally:
        O.set_threads(1)
    assert np.array_equal(ra, rb) and ra.mean() > 0.05
    ratio = np.abs(a.v - b.v) / (1e-5 * np.maximum(np.abs(a.v), 1.0))
    assert ratio.max() > 1.5, ratio.max()
    assert np.quantile(ratio, 0.99) < 1.0


def test_synaptic_sum_order_fp32():
    """The float32 mirror adds a step's arrivals oldest spike first (largest
    delay first, then pre-neuron): into neuron 3 at step 2 arrive +1e8 and +1
    (delay 2, from neurons 0 and 1, spiking at step 0) and -1e8 (delay 1, from
    neuron 2, spiking at step 1).  Oldest first, (1e8 + 1) - 1e8 = 0 in
    float32; in ascending delay order it would be (-1e8 + 1e8) + 1 = 1;
    float64 gives 1 either way."""
    wl = W._base(4, "f32", [0.5, 0.5, 0.5, 1e30], 0.0, 0.0, 0, 2, 3)
    wl.update(pre=np.array([0, 1, 2], np.int32), post=np.array([3, 3, 3], np.int32),
              weight=np.array([1e8, 1.0, -1e8]), delay=np.array([2, 2, 1], np.int32))
    wl["events"] = dict(step=np.array([0, 0, 1], np.int32), neuron=np.array([0, 1, 2], np.int32),
                        value=np.ones(3))
    st32, r32, _ = O.run(wl, O.F32, 3, record_v=True)
    st64, r64, _ = O.run(wl, O.F64, 3, record_v=True)
    assert r32[0, :2].tolist() == [1, 1] and r32[1, 2] == 1
    assert st32.ctrace[2, 3] == 0.0 and st64.ctrace[2, 3] == 1.0
