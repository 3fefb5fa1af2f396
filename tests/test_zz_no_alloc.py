"""sn_run_dense_noalloc: the dense run for callers that cannot allocate device
memory (an application whose device memory is all owned by its own pool
allocator, or a plug-in whose host does not let it allocate).  It runs the same
kernel as the ordinary dense entry point (sn_create_dense + sn_run), so its
raster and state must equal that entry point's bit for bit on the same network
and input, on two calls in a row that share the library's fixed scratch
array."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def test_noalloc_matches_dense_entry_point_twice():
    from paper_2305_02510_gb300 import sn as S, workloads as W
    wl = W.large_dense(n=1500, steps=150)
    n, T = wl["n"], 150
    # the ordinary entry point
    ctx = S.from_workload(wl, record_steps=T)
    S.sn_run(ctx, T)
    S.sn_sync(ctx)
    want = S.sn_get_spikes(ctx, 0, T)
    v_want, r_want = S.sn_get_state(ctx)
    assert S.unpack_raster(want, n).sum() > 0
    # the same network on caller-owned device tensors
    dev = torch.device("cuda")
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev)
    w = f32(wl["dense_w"])
    th, lk, rs = f32(wl["threshold"]), f32(wl["leak"]), f32(wl["reset"])
    R = torch.tensor(wl["refractory"], dtype=torch.int32, device=dev)
    po = wl["poisson"]
    thr = np.zeros(n, np.uint32)
    amp = np.zeros(n, np.float32)
    # per-neuron threshold floor(rate * 2^32) of the float32 rate, as the ABI states
    thr[po["neuron"]] = np.floor(np.float64(np.float32(po["rate"])) * 4294967296.0).astype(np.uint32)
    amp[po["neuron"]] = po["amplitude"]
    pthr = torch.tensor(thr.view(np.int32), device=dev)
    pamp = torch.tensor(amp, device=dev)
    words = (n + 31) // 32
    for call in range(2):
        v = rs.clone()
        r = torch.zeros(n, dtype=torch.int32, device=dev)
        raster = torch.full((T, words), -1, dtype=torch.int32, device=dev)
        S.sn_run_dense_noalloc(n, wl["dense_delay"], T, w, th, lk, rs, R, v, r, raster,
                               pthr, pamp, po["seed"])
        got = raster.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), f"call {call}: raster differs from sn_run"
        # the same kernel on the same input: the state is bit-identical
        assert np.array_equal(v.cpu().numpy().view(np.uint32), np.asarray(v_want, np.float32).view(np.uint32)), \
            f"call {call}: state differs from sn_run"
        assert np.array_equal(r.cpu().numpy(), r_want)


def test_noalloc_binding_rejects_short_and_host_buffers():
    """The binding refuses buffers the kernel would read or write past their
    end before any C call."""
    from paper_2305_02510_gb300 import sn as S
    n, T = 64, 4
    dev = torch.device("cuda")
    f = lambda k: torch.zeros(k, device=dev)
    i = lambda k: torch.zeros(k, dtype=torch.int32, device=dev)
    good = dict(w=f(n * n), threshold=f(n), leak=f(n), reset=f(n), refractory=i(n), v=f(n), r=i(n),
                raster=i(T * 2))
    S.sn_run_dense_noalloc(n, 1, T, **good)
    for k, bad in (("w", f(n * n - 1)), ("v", f(n - 1)), ("r", f(n)), ("raster", i(T * 2 - 1)),
                   ("threshold", np.zeros(n, np.float32)), ("leak", f(2 * n)[::2])):
        with pytest.raises(ValueError):
            S.sn_run_dense_noalloc(n, 1, T, **{**good, k: bad})
