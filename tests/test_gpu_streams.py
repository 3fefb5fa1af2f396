"""Setters are ordered after the work already queued on a context's stream.

A context may run on a stream created with cudaStreamNonBlocking (every torch
stream is one), which a blocking cudaMemcpy on the legacy default stream does
not wait for.  sn_run only queues its kernel, so a setter called right after it
must not overwrite the Poisson table or the event list while that kernel still
reads them.  The trajectory of run(T1), set new input, run(T2) on such a stream
must equal the oracle's run with the first input for T1 steps and the second
after, bit for bit (integer network)."""

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


@pytest.mark.parametrize("pull", [False, True])
def test_setters_after_queued_run_on_nonblocking_stream(pull):
    from paper_2305_02510_gb300 import sn as S
    T1, T2 = 400, 60
    wl = W.large_sparse(integer=True, n=20_000, steps=T1 + T2)
    n = wl["n"]
    stream = torch.cuda.Stream()          # created with cudaStreamNonBlocking
    ctx = S.from_workload(wl, flags=S.SN_PROP_PULL if pull else S.SN_AUTO, record_steps=T1 + T2,
                          stream=stream.cuda_stream)
    po = wl["poisson"]
    seed2 = int(po["seed"]) ^ 0x5A5A
    rng = np.random.default_rng(11)
    ev2 = {"step": rng.integers(T1, T1 + T2, 400).astype(np.int32),
           "neuron": rng.integers(0, n, 400).astype(np.int32),
           "value": np.full(400, 21.0, np.float32)}
    S.sn_run(ctx, T1)                      # queued, still running when the setters below start
    S.sn_set_poisson(ctx, po["neuron"], po["rate"], po["amplitude"], seed2)
    S.sn_set_input(ctx, ev2["step"], ev2["neuron"], ev2["value"])
    S.sn_run(ctx, T2)
    S.sn_sync(ctx)
    raster = S.unpack_raster(S.sn_get_spikes(ctx, 0, T1 + T2), n)
    v, r = S.sn_get_state(ctx)
    # the oracle: first input for T1 steps, then the new seed and events
    st1, want1, _ = O.run(wl, O.INT, T1)
    assert np.array_equal(raster[:T1], want1), "first segment differs from the oracle"
    wl2 = dict(wl, events=ev2)
    compare.check_int_run(wl2, raster[T1:], v, r, T2, state=st1, poisson_seed=seed2)
    assert raster[T1:].sum() > 0
