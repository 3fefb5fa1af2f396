"""sn_run_dense_noalloc: the dense run for callers that cannot allocate device
memory (for example code running during CUDA stream capture, where cudaMalloc
is not allowed, or an application whose device memory is all owned by its own
pool).  Its output must match the ordinary dense entry point (sn_create_dense
+ sn_run) on the same network and input, on two calls in a row that share
the library's fixed scratch array."""

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
    theta = np.asarray(np.float32(wl["threshold"]), np.float64)
    for call in range(2):
        v = rs.clone()
        r = torch.zeros(n, dtype=torch.int32, device=dev)
        raster = torch.full((T, words), -1, dtype=torch.int32, device=dev)
        S.sn_run_dense_noalloc(n, wl["dense_delay"], T, w, th, lk, rs, R, v, r, raster,
                               pthr, pamp, po["seed"])
        got = raster.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), f"call {call}: raster differs from sn_run"
        vv = v.cpu().numpy().astype(np.float64)
        tol = 1e-5 * np.maximum(np.abs(v_want.astype(np.float64)), np.abs(theta))
        assert np.all(np.abs(vv - v_want) <= tol), f"call {call}: state differs"
        assert np.array_equal(r.cpu().numpy(), r_want)


def test_noalloc_rejects_oversized_network():
    from paper_2305_02510_gb300 import sn as S
    n = 4096
    dev = torch.device("cuda")
    z = torch.zeros(n, device=dev)
    R = torch.zeros(n, dtype=torch.int32, device=dev)
    w = torch.zeros(1, device=dev)    # never read: the size check comes first
    raster = torch.zeros(1, dtype=torch.int32, device=dev)
    # delay 64 needs 66 * 4 * n bytes of ring per 4096 neurons: too much scratch
    # only for large n; at n = 4096 it fits, at n = 70000 it does not
    with pytest.raises(S.SnError) as e:
        S.sn_run_dense_noalloc(70000, 64, 1, w, z, z, z, R, z, R, raster)
    assert e.value.status == S.SN_EINVAL
