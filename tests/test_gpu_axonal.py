"""Axonal delays (Section 2.2: a neuron parameter beside threshold, leak and
refractory period) through sn_create_axonal: integer networks bit-exact
against the oracle in both propagation modes, float networks within the
float rules, and argument checks."""

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


def with_axonal(wl, seed, amax):
    rng = np.random.default_rng(seed)
    ax = rng.integers(0, amax + 1, wl["n"]).astype(np.int32)
    wl = dict(wl, axonal_delay=ax)
    wl["max_delay"] = int(wl["max_delay"]) + amax
    return wl


@pytest.mark.parametrize("prop", ["push", "pull"])
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_axonal_int_bit_exact(seed, prop):
    from paper_2305_02510_gb300 import sn as S
    wl = with_axonal(W.random_small(100 + seed, n=300, integer=True, steps=200, max_delay=4, p=0.05,
                                    events_rate=1.0), seed, 5)
    ctx = S.from_workload(wl, record_steps=200)
    S.sn_set_propagation(ctx, S.SN_PULL if prop == "pull" else S.SN_PUSH)
    S.sn_run(ctx, 200)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 200), wl["n"])
    v, r = S.sn_get_state(ctx)
    compare.check_int_run(wl, raster, v, r, 200)
    assert raster.sum() > 0


def test_axonal_float_large():
    from paper_2305_02510_gb300 import sn as S
    wl = with_axonal(W.large_sparse(n=20000, k=50, steps=150), 7, 3)
    ctx = S.from_workload(wl, record_steps=150)
    S.sn_run(ctx, 150)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 150), wl["n"])
    v, r = S.sn_get_state(ctx)
    compare.check_float_run(wl, raster, v, r, 150)
    assert raster.sum() > 0


def test_axonal_argument_checks():
    from paper_2305_02510_gb300 import sn as S
    wl = W.random_small(9, n=20, integer=True, steps=10, max_delay=3)
    for bad in (np.full(20, -1), np.full(20, 3)):      # negative; delay + axonal > max_delay
        with pytest.raises(S.SnError) as e:
            S.sn_create(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], wl["pre"], wl["post"],
                        wl["weight"], wl["delay"], dtype=S.SN_I32, max_delay=3, axonal_delay=bad)
        assert e.value.status == S.SN_EINVAL
