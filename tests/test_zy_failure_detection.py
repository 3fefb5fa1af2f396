"""Failure detection on the GPU without a fault: a grid barrier that one
block never reaches runs out after its wall-clock bound, the waiting blocks
latch SN_ETIMEOUT and return, and the CUDA context stays usable (a small
network then runs bit-exact against the oracle)."""

import time

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


def test_barrier_wait_runs_out_and_context_stays_usable():
    from paper_2305_02510_gb300 import sn as S
    t0 = time.monotonic()
    st = S.sn_selftest_barrier_timeout()
    dt = time.monotonic() - t0
    assert st == S.SN_ETIMEOUT
    assert 1.5 < dt < 60.0, dt                 # the bound is 2 s of wall-clock time
    wl = W.tiny(integer=True)
    ctx = S.from_workload(wl, record_steps=300)
    S.sn_run(ctx, 300)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, 300), wl["n"])
    v, r = S.sn_get_state(ctx)
    compare.check_int_run(wl, raster, v, r, 300)
