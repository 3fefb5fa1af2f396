"""The C ABI without a GPU: libsn.so loads, exports every entry point that
include/sn.h declares, and rejects bad arguments with SN_EINVAL before any
CUDA call is made."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    from paper_2305_02510_gb300 import build, sn
    build.build()
    sn.lib()
    return sn


def declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:sn_status|const char\s*\*|void|int32_t)\s*\*?\s*(sn_\w+)\s*\(",
                                txt, re.M)
    return names


def test_exports_every_declared_symbol(S):
    names = declared()
    assert "sn_create" in names and "sn_run" in names and len(names) >= 17
    missing = [n for n in names if not hasattr(S.lib(), n)]
    assert not missing


def _neurons(S, n, keep):
    th, lk, rs = np.ones(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.float32)
    rf = np.zeros(n, np.int32)
    keep += [th, lk, rs, rf]
    nr = S.sn_neurons()
    nr.n = n
    nr.threshold, nr.leak, nr.reset, nr.refractory = (a.ctypes.data for a in (th, lk, rs, rf))
    return nr, (th, lk, rs, rf)


def _create(S, n=4, pre=(0,), post=(1,), w=(1.0,), d=(1,), dtype=0, D=2, flags=0, leak=None):
    keep = []
    nr, arrs = _neurons(S, n, keep)
    if leak is not None:
        arrs[1][:] = leak
    pre, post = np.array(pre, np.int32), np.array(post, np.int32)
    w, d = np.array(w, np.float32), np.array(d, np.int32)
    sy = S.sn_synapses()
    sy.m = pre.size
    sy.pre, sy.post, sy.weight, sy.delay = pre.ctypes.data, post.ctypes.data, w.ctypes.data, d.ctypes.data
    cfg = S.sn_config()
    cfg.dtype, cfg.max_delay, cfg.flags, cfg.record_steps = dtype, D, flags, 0
    h = C.c_void_p()
    st = S.lib().sn_create(C.byref(cfg), C.byref(nr), C.byref(sy), C.byref(h))
    return st, S.lib().sn_last_error(None).decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(d=(3,)), "delay"),
    (dict(d=(0,)), "delay"),
    (dict(pre=(4,)), "index"),
    (dict(post=(-1,)), "index"),
    (dict(w=(float("nan"),)), "weight"),
    (dict(w=(0.5,), dtype=1), "integer"),
    (dict(D=0), "max_delay"),
    (dict(D=65), "max_delay"),
    (dict(dtype=7), "dtype"),
    (dict(flags=3), "exclusive"),
    (dict(flags=64), "flags"),
    (dict(leak=-1.0), "leak"),
    (dict(n=0), "n must"),
])
def test_invalid_arguments(S, kw, frag):
    st, msg = _create(S, **kw)
    assert st == S.SN_EINVAL
    assert frag in msg


def test_version_and_null_handles(S):
    L = S.lib()
    assert b"sm_103a" in L.sn_version()
    assert L.sn_run(None, 1) == S.SN_EINVAL
    assert L.sn_sync(None) == S.SN_EINVAL
    assert L.sn_set_propagation(None, S.SN_PULL) == S.SN_EINVAL
    assert L.sn_get_propagation(None, None) == S.SN_EINVAL
    assert L.sn_selftest_barrier_timeout(None, None) == S.SN_EINVAL
    L.sn_destroy(None)


def test_new_entry_points_reject_bad_arguments(S):
    """sn_set_weights, sn_ff_set_engine and sn_create_axonal validate their
    arguments before any CUDA call."""
    L = S.lib()
    assert L.sn_set_weights(None, None, 0) == S.SN_EINVAL
    assert L.sn_ff_set_engine(None, S.SN_FF_TENSOR) == S.SN_EINVAL
    keep = []
    n = 4
    nr, _ = _neurons(S, n, keep)
    pre, post = np.array([0, 1], np.int32), np.array([1, 2], np.int32)
    w, d = np.array([1.0, 1.0], np.float32), np.array([1, 2], np.int32)
    sy = S.sn_synapses()
    sy.m = 2
    sy.pre, sy.post, sy.weight, sy.delay = pre.ctypes.data, post.ctypes.data, w.ctypes.data, d.ctypes.data
    cfg = S.sn_config()
    cfg.dtype, cfg.max_delay, cfg.flags, cfg.record_steps = 0, 3, 0, 0
    h = C.c_void_p()
    for ax, frag in (([0, 2, 0, 0], "axonal"), ([-1, 0, 0, 0], "axonal"), ([3, 0, 0, 0], "axonal")):
        a = np.array(ax, np.int32)
        st = L.sn_create_axonal(C.byref(cfg), C.byref(nr), C.byref(sy), a.ctypes.data, C.byref(h))
        assert st == S.SN_EINVAL, ax
        assert frag in L.sn_last_error(None).decode()


def _shared(S, n=128, trains=128, dtype=1, D=1, wval=0):
    keep = []
    nr, _ = _neurons(S, n, keep)
    w = np.full((n, n), wval, np.int8)
    cfg = S.sn_config()
    cfg.dtype, cfg.max_delay, cfg.flags, cfg.record_steps = dtype, D, 0, 0
    h = C.c_void_p()
    st = S.lib().sn_create_shared_dense_i8(C.byref(cfg), C.byref(nr), w.ctypes.data, trains, C.byref(h))
    return st, S.lib().sn_last_error(None).decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(n=100), "multiple of 128"),
    (dict(trains=100), "trains"),
    (dict(dtype=0), "SN_I32"),
    (dict(D=2), "delay 1"),
    (dict(wval=9), "-8 .. 8"),
    (dict(wval=-9), "-8 .. 8"),
])
def test_shared_dense_rejects_bad_arguments(S, kw, frag):
    st, msg = _shared(S, **kw)
    assert st == S.SN_EINVAL and frag in msg, msg


def _batch(S, sizes=(4, 5), D=2, delay=1, dtype=0):
    keep = []
    nrs = (S.sn_neurons * max(1, len(sizes)))()
    sys_ = (S.sn_synapses * max(1, len(sizes)))()
    for b, n in enumerate(sizes):
        nr, _ = _neurons(S, n, keep)
        nrs[b] = nr
        pre, post = np.array([0], np.int32), np.array([min(1, n - 1)], np.int32)
        w, d = np.array([1.0], np.float32), np.array([delay], np.int32)
        keep += [pre, post, w, d]
        sy = S.sn_synapses()
        sy.m = 1
        sy.pre, sy.post, sy.weight, sy.delay = pre.ctypes.data, post.ctypes.data, w.ctypes.data, d.ctypes.data
        sys_[b] = sy
    cfg = S.sn_config()
    cfg.dtype, cfg.max_delay, cfg.flags, cfg.record_steps = dtype, D, 0, 0
    h = C.c_void_p()
    st = S.lib().sn_create_batch(C.byref(cfg), len(sizes), nrs, sys_, C.byref(h))
    return st, S.lib().sn_last_error(None).decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(sizes=()), "nets"),
    (dict(sizes=(4, 5000)), "1..4096"),
    (dict(D=17), "max_delay"),
    (dict(delay=3), "delay"),
    (dict(dtype=5), "dtype"),
])
def test_batch_rejects_bad_arguments(S, kw, frag):
    st, msg = _batch(S, **kw)
    assert st == S.SN_EINVAL and frag in msg, msg


def _ff(S, sizes=(3, 4, 2), k=10, batch=2, steps=10, delay=1, layers=None):
    sz = np.array(sizes, np.int32)
    L = len(sizes) - 1 if layers is None else layers
    ds = [np.full((max(1, sizes[l]), max(1, sizes[l + 1])), delay, np.uint8) for l in range(len(sizes) - 1)]
    ptrs = (C.c_void_p * max(1, len(ds)))(*[d.ctypes.data for d in ds])
    p = S.sn_ff_params(1.0, 0.05, 0.0, 0, 10.0, k)
    cfg = S.sn_config()
    cfg.dtype, cfg.max_delay, cfg.flags, cfg.record_steps = 0, 1, 0, 0
    h = C.c_void_p()
    st = S.lib().sn_create_ff(C.byref(cfg), L, sz.ctypes.data, ptrs, C.byref(p), batch, steps, C.byref(h))
    return st, S.lib().sn_last_error(None).decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(layers=0), "layers"),
    (dict(layers=17), "layers"),
    (dict(k=3), "checkpoint_every"),
    (dict(delay=5), "delays"),
    (dict(delay=0), "delays"),
    (dict(batch=0), "batch"),
    (dict(steps=0), "steps"),
    (dict(sizes=(3, 0, 2)), "sizes"),
])
def test_ff_rejects_bad_arguments(S, kw, frag):
    st, msg = _ff(S, **kw)
    assert st == S.SN_EINVAL and frag in msg, msg


def _noalloc(S, **kw):
    a = S.sn_dense_noalloc_args()
    a.n, a.delay, a.steps = 8, 1, 4
    for name in ("w", "threshold", "leak", "reset", "refractory", "v", "r", "raster"):
        setattr(a, name, 256)               # never dereferenced by the checks
    for k, v in kw.items():
        setattr(a, k, v)
    return S.lib().sn_run_dense_noalloc(C.byref(a))


@pytest.mark.parametrize("kw", [dict(n=0), dict(n=200001), dict(delay=0), dict(delay=65), dict(steps=-1),
                                dict(w=None), dict(v=None), dict(raster=None),
                                dict(poisson_threshold=256), dict(poisson_amplitude=256)])
def test_noalloc_rejects_bad_arguments(S, kw):
    assert _noalloc(S, **kw) == S.SN_EINVAL


def test_noalloc_zero_steps_is_a_no_op(S):
    """Zero steps return SN_OK before any CUDA call (and need no raster)."""
    assert _noalloc(S, steps=0, raster=None) == S.SN_OK
    assert S.lib().sn_run_dense_noalloc(None) == S.SN_EINVAL


def test_noalloc_rejects_oversized_scratch_before_any_cuda_call(S):
    """The scratch need depends only on n and delay, so a network beyond the
    fixed array is refused (with the sizes in the message) before any CUDA
    call: here with dummy pointers and no GPU."""
    # 70,000 neurons at delay 64: about 65 * 4 * 70000 bytes of ring, over 16 MiB
    assert _noalloc(S, n=70000, delay=64) == S.SN_EINVAL
    msg = S.lib().sn_last_error(None).decode()
    assert "scratch" in msg and str(16 << 20) in msg, msg
    # the largest delay that fits 200,000 neurons is accepted by the check
    # (zero steps: nothing runs)
    assert _noalloc(S, n=200000, delay=18, steps=0, raster=None) == S.SN_OK
    assert _noalloc(S, n=200000, delay=19, steps=0, raster=None) == S.SN_EINVAL


def test_noalloc_binding_rejects_host_arrays(S):
    """The binding wants CUDA tensors: numpy arrays (host pointers the kernel
    would dereference) raise ValueError before the C call."""
    n = 8
    z = np.zeros(n, np.float32)
    zi = np.zeros(n, np.int32)
    with pytest.raises(ValueError):
        S.sn_run_dense_noalloc(n, 1, 2, np.zeros(n * n, np.float32), z, z, z, zi, z.copy(), zi.copy(),
                               np.zeros(2, np.int32))


def _dense(S, n=4, delay=1, D=2, dtype=0, wval=0.5, flags=0):
    keep = []
    nr, _ = _neurons(S, n, keep)
    w = np.full((max(n, 1), max(n, 1)), wval, np.float32)
    cfg = S.sn_config()
    cfg.dtype, cfg.max_delay, cfg.flags, cfg.record_steps = dtype, D, flags, 0
    h = C.c_void_p()
    st = S.lib().sn_create_dense(C.byref(cfg), C.byref(nr), w.ctypes.data, delay, C.byref(h))
    return st, S.lib().sn_last_error(None).decode()


@pytest.mark.parametrize("kw,status,frag", [
    (dict(dtype=1), "SN_EUNSUPPORTED", "SN_F32"),
    (dict(flags=4), "SN_EUNSUPPORTED", "SN_PROP_PULL"),
    (dict(n=0), "SN_EINVAL", "dense n"),
    (dict(delay=0), "SN_EINVAL", "delay"),
    (dict(delay=3), "SN_EINVAL", "delay"),
    (dict(wval=float("inf")), "SN_EINVAL", "weight"),
    (dict(flags=3 << 8), "SN_EINVAL", "SN_DENSE_SLAB"),
    (dict(flags=64 << 8), "SN_EINVAL", "flags"),
    (dict(flags=0x1000), "SN_EUNSUPPORTED", "SN_PULL_"),
    (dict(flags=0x3000), "SN_EINVAL", "exclusive"),
])
def test_dense_rejects_bad_arguments(S, kw, status, frag):
    st, msg = _dense(S, **kw)
    assert st == getattr(S, status) and frag in msg, (st, msg)


def test_binding_neuron_arrays(S):
    """The binding repeats a single parameter value n times and refuses
    arrays of different lengths before any C call."""
    keep = []
    nr = S._neurons(np.ones(5), 0.1, [0.0], 2, keep)
    assert nr.n == 5
    lk = keep[1]
    assert lk.size == 5 and np.all(lk == np.float32(0.1)) and np.all(keep[3] == 2)
    with pytest.raises(ValueError):
        S._neurons(np.ones(5), np.zeros(4), 0.0, 0, [])


def test_binding_synapse_and_input_arrays(S):
    """Synapse, input-event and Poisson arrays: pre and post must pair up,
    weights and delays (event values, rates, amplitudes) match or are single
    values; everything is checked before a C call (no GPU needed here)."""
    keep = []
    pre, post, w, d = S._synapses([0, 1, 2], [1, 2, 0], 0.5, [1, 2, 3], keep)
    assert w.tolist() == [0.5] * 3 and d.tolist() == [1, 2, 3]
    for bad in (([0, 1], [1], 1.0, 1), ([0, 1], [1, 0], [1.0, 2.0, 3.0], 1), ([0, 1], [1, 0], 1.0, [1, 2, 3])):
        with pytest.raises(ValueError):
            S._synapses(*bad, [])
    dummy = S.Ctx(None, 4, 0, 1, "sparse", 0)
    with pytest.raises(ValueError):
        S.sn_set_input(dummy, [0, 1], [0], [1.0, 1.0])
    with pytest.raises(ValueError):
        S.sn_set_input(dummy, [0, 1], [0, 1], [1.0, 1.0, 1.0])
    with pytest.raises(ValueError):
        S.sn_set_poisson(dummy, [0, 1, 2], [0.1, 0.2], 1.0, 7)
    with pytest.raises(ValueError):
        S.sn_create_dense(np.ones(3), 0.0, 0.0, 0, np.zeros(8, np.float32))


def test_binding_output_buffers(S):
    """Caller-provided output buffers must be contiguous and large enough
    for what the library writes; checked before the C call."""
    dummy = S.Ctx(None, 40, 0, 2, "sparse", 10)
    with pytest.raises(ValueError):
        S.sn_get_spikes(dummy, 0, 5, out=np.zeros((4, 2), np.uint32))
    with pytest.raises(ValueError):
        S.sn_get_spikes(dummy, 0, 5, out=np.zeros((5, 4), np.uint32)[:, ::2])
    with pytest.raises(ValueError):
        S.sn_get_state(dummy, v=np.zeros(39, np.float32))
    with pytest.raises(ValueError):
        S.sn_get_state(dummy, refractory=np.zeros(10, np.int32))
    with pytest.raises(ValueError):
        S.sn_get_weights(dummy, out=np.zeros(9, np.float32))
    with pytest.raises(ValueError):
        S.sn_get_trace(dummy, out=np.zeros(3, np.float32))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        S._out(torch.zeros(3), 16, "x")
    assert S._out(torch.zeros(4), 16, "x") is not None


def test_binding_ff_arguments(S):
    """Feedforward contexts: one delay array of n_in x n_out per layer at
    creation, and CUDA tensors of the exact sizes and dtypes for the forward
    and backward, checked before any C call."""
    with pytest.raises(ValueError):
        S.sn_create_ff([3, 4, 2], [np.ones((3, 4), np.uint8)], threshold=1, leak=0, reset=0, refractory=0,
                       slope=10, checkpoint_every=10, batch=2, steps=10)
    with pytest.raises(ValueError):
        S.sn_create_ff([3, 4], [np.ones((3, 5), np.uint8)], threshold=1, leak=0, reset=0, refractory=0,
                       slope=10, checkpoint_every=10, batch=2, steps=10)
    dummy = S.Ctx(None, 2, 0, 0, "ff", 0)
    dummy.sizes, dummy.batch, dummy.steps, dummy.k = [3, 4, 2], 2, 10, 10
    with pytest.raises(ValueError):                     # host arrays are not CUDA tensors
        S.sn_ff_forward(dummy, np.zeros((10, 2, 3), np.uint8), [np.zeros((3, 4), np.float32)] * 2,
                        np.zeros((2, 2), np.float32))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        S._dev(torch.zeros(6), 6, "float32", "x")      # a CPU tensor
