"""Thin Python binding of libsn.so: the entry points of include/sn.h under the
same names, with argument marshalling only.

Host arrays are numpy arrays; device buffers are torch CUDA tensors (their
data pointers are passed through).  Every call raises SnError when the C call
returns a status other than SN_OK.  The library is loaded on first use, and
loading fails loudly if it has not been built: there is no fallback path.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SN_OK, SN_EINVAL, SN_ENOMEM, SN_ECUDA, SN_ESTATE, SN_ETIMEOUT, SN_EUNSUPPORTED, SN_EOVERFLOW = range(8)
SN_F32, SN_I32 = 0, 1
SN_AUTO, SN_EXEC_CTA, SN_EXEC_GRID, SN_PROP_PULL, SN_FF_RECOMPUTE = 0, 1, 2, 4, 8
SN_PUSH, SN_PULL = 0, 1
SN_PULL_PLAIN, SN_PULL_CODED = 0x1000, 0x2000


def SN_DENSE_SLAB(k: int) -> int:
    """sn_create_dense flag: column slabs of 32 * k columns per block (k = 1, 2, 4, 8)."""
    return int(k) << 8

SN_FF_AUTO, SN_FF_SIMT, SN_FF_TENSOR = 0, 1, 2
_NAMES = ["SN_OK", "SN_EINVAL", "SN_ENOMEM", "SN_ECUDA", "SN_ESTATE", "SN_ETIMEOUT",
          "SN_EUNSUPPORTED", "SN_EOVERFLOW"]


class SnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_NAMES[status] if 0 <= status < len(_NAMES) else status}: {msg}")
        self.status = status


class sn_config(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("max_delay", C.c_int32), ("flags", C.c_uint32),
                ("record_steps", C.c_int32), ("cuda_stream", C.c_void_p)]


class sn_neurons(C.Structure):
    _fields_ = [("n", C.c_int32), ("threshold", C.c_void_p), ("leak", C.c_void_p),
                ("reset", C.c_void_p), ("refractory", C.c_void_p)]


class sn_synapses(C.Structure):
    _fields_ = [("m", C.c_int64), ("pre", C.c_void_p), ("post", C.c_void_p),
                ("weight", C.c_void_p), ("delay", C.c_void_p)]


class sn_dense_noalloc_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("delay", C.c_int32), ("steps", C.c_int32), ("pad", C.c_int32),
                ("w", C.c_void_p), ("threshold", C.c_void_p), ("leak", C.c_void_p),
                ("reset", C.c_void_p), ("refractory", C.c_void_p),
                ("poisson_threshold", C.c_void_p), ("poisson_amplitude", C.c_void_p),
                ("seed", C.c_uint64), ("v", C.c_void_p), ("r", C.c_void_p),
                ("raster", C.c_void_p), ("cuda_stream", C.c_void_p)]


class sn_ff_params(C.Structure):
    _fields_ = [("threshold", C.c_float), ("leak", C.c_float), ("reset", C.c_float),
                ("refractory", C.c_int32), ("surrogate_slope", C.c_float), ("checkpoint_every", C.c_int32)]


_lib = None
_lock = threading.Lock()
_P = C.c_void_p


def lib():
    """Load libsn.so (raises if it is missing: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libsn.so not built ({_build.LIB}); run "
                                   "paper_2305_02510_gb300.build.build() first")
            L = C.CDLL(_build.LIB)
            sig = {
                "sn_create": [C.POINTER(sn_config), C.POINTER(sn_neurons), C.POINTER(sn_synapses),
                              C.POINTER(_P)],
                "sn_create_dense": [C.POINTER(sn_config), C.POINTER(sn_neurons), _P, C.c_int32,
                                    C.POINTER(_P)],
                "sn_create_axonal": [C.POINTER(sn_config), C.POINTER(sn_neurons), C.POINTER(sn_synapses), _P,
                                     C.POINTER(_P)],
                "sn_create_shard": [C.POINTER(sn_config), C.POINTER(sn_neurons), C.POINTER(sn_synapses),
                                    C.c_int32, C.c_int32, C.POINTER(_P)],
                "sn_shard_info": [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
                "sn_shard_put_spikes": [_P, C.c_int64, C.c_int64, _P, C.c_int32],
                "sn_create_batch": [C.POINTER(sn_config), C.c_int32, C.POINTER(sn_neurons),
                                    C.POINTER(sn_synapses), C.POINTER(_P)],
                "sn_batch_config": [_P, C.c_int32, C.c_int32],
                "sn_autotune": [_P, C.c_int32, C.POINTER(C.c_float)],
                "sn_create_shared_dense_i8": [C.POINTER(sn_config), C.POINTER(sn_neurons), _P, C.c_int32,
                                              C.POINTER(_P)],
                "sn_create_ff": [C.POINTER(sn_config), C.c_int32, _P, _P, C.POINTER(sn_ff_params), C.c_int32,
                                 C.c_int32, C.POINTER(_P)],
                "sn_ff_forward": [_P, _P, _P, _P],
                "sn_backward": [_P, _P, _P, C.c_int32],
                "sn_ff_get_spikes": [_P, C.c_int32, _P, C.c_int32],
                "sn_ff_set_engine": [_P, C.c_int32],
                "sn_ff_get_checkpoints": [_P, C.c_int32, _P, C.c_int32],
                "sn_set_input": [_P, C.c_int64, _P, _P, _P],
                "sn_set_poisson": [_P, C.c_int32, _P, _P, _P, C.c_uint64],
                "sn_set_poisson_stream": [_P, C.c_int32, _P, _P, _P, C.c_uint64, C.c_uint64],
                "sn_stdp": [_P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32],
                "sn_run": [_P, C.c_int32],
                "sn_reset": [_P],
                "sn_sync": [_P],
                "sn_get_spikes": [_P, C.c_int64, C.c_int64, _P, C.c_int32],
                "sn_get_state": [_P, _P, _P, C.c_int32],
                "sn_get_trace": [_P, _P, C.c_int32],
                "sn_get_weights": [_P, _P, C.c_int32],
                "sn_set_weights": [_P, _P, C.c_int32],
                "sn_get_counters": [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)],
                "sn_set_propagation": [_P, C.c_int32],
                "sn_get_propagation": [_P, C.POINTER(C.c_int32)],
                "sn_pull_store_info": [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
                "sn_save": [_P, _P, C.POINTER(C.c_size_t)],
                "sn_load": [_P, _P, C.c_size_t],
                "sn_selftest_barrier_timeout": [_P, C.POINTER(C.c_int32)],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.sn_run_dense_noalloc.argtypes = [C.POINTER(sn_dense_noalloc_args)]
            L.sn_run_dense_noalloc.restype = C.c_int
            L.sn_last_error.argtypes = [_P]
            L.sn_last_error.restype = C.c_char_p
            L.sn_destroy.argtypes = [_P]
            L.sn_destroy.restype = None
            L.sn_version.argtypes = []
            L.sn_version.restype = C.c_char_p
            _lib = L
    return _lib


def _check(st, ctx=None):
    if st != SN_OK:
        msg = lib().sn_last_error(ctx.handle if ctx is not None else None)
        raise SnError(st, msg.decode() if msg else "")


def _arr(a, dt):
    return np.ascontiguousarray(np.asarray(a), dtype=dt)


def _ptr(x):
    """Data pointer of a numpy array or a torch tensor (None for None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _is_dev(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _out(x, nbytes, what):
    """A caller's output buffer (numpy array or torch tensor) must be
    contiguous and hold at least nbytes: the library writes that many."""
    if hasattr(x, "data_ptr"):
        size, contig = x.numel() * x.element_size(), x.is_contiguous()
    else:
        size, contig = x.nbytes, x.flags["C_CONTIGUOUS"]
    if not contig or size < nbytes:
        raise ValueError(f"{what}: need a contiguous buffer of {nbytes} bytes, got {size}"
                         f"{'' if contig else ' (not contiguous)'}")
    return x


class Ctx:
    """Owns one sn_ctx handle; n, dtype and kind are kept for output sizing."""

    def __init__(self, handle, n, dtype, words, kind, m):
        self.handle = handle
        self.n, self.dtype, self.words, self.kind, self.m = n, dtype, words, kind, m

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sn_destroy(self.handle)
            self.handle = None


def _config(dtype, max_delay, flags, record_steps, stream):
    cfg = sn_config()
    cfg.dtype = SN_I32 if dtype in (SN_I32, "i32") else SN_F32
    cfg.max_delay = int(max_delay)
    cfg.flags = int(flags)
    cfg.record_steps = int(record_steps)
    cfg.cuda_stream = stream
    return cfg


def _match(what, n, *arrs):
    """Arrays of n values each (the C side reads n of each); a single value
    is repeated n times, any other length raises ValueError."""
    out = []
    for a in arrs:
        a = a.reshape(-1)
        if a.size == n:
            out.append(a)
        elif a.size == 1 and n != 1:
            out.append(np.full(n, a[0], a.dtype))
        else:
            raise ValueError(f"{what}: expected {n} values, got {a.size}")
    return out


def _synapses(pre, post, weight, delay, keep):
    pre, post = _arr(pre, np.int32).reshape(-1), _arr(post, np.int32).reshape(-1)
    if pre.size != post.size:
        raise ValueError(f"synapses: {pre.size} pre and {post.size} post indices")
    w, d = _match("synapse weights and delays", pre.size, _arr(weight, np.float32), _arr(delay, np.int32))
    keep += [pre, post, w, d]
    return pre, post, w, d


def _neurons(threshold, leak, reset, refractory, keep):
    """Neuron parameter arrays of one size n; a single value is repeated n
    times (the C side always reads n values of each)."""
    arrs = [_arr(threshold, np.float32), _arr(leak, np.float32), _arr(reset, np.float32),
            _arr(refractory, np.int32)]
    th, lk, rs, rf = _match("neuron parameters", max(a.size for a in arrs), *arrs)
    keep += [th, lk, rs, rf]
    nr = sn_neurons()
    nr.n = th.size
    nr.threshold, nr.leak, nr.reset, nr.refractory = _ptr(th), _ptr(lk), _ptr(rs), _ptr(rf)
    return nr


def sn_create(threshold, leak, reset, refractory, pre, post, weight, delay, *, dtype=SN_F32,
              max_delay=None, flags=SN_AUTO, record_steps=0, stream=None, axonal_delay=None) -> Ctx:
    """sn_create, or sn_create_axonal when axonal_delay (n values) is given."""
    keep = []
    nr = _neurons(threshold, leak, reset, refractory, keep)
    pre, post, w, d = _synapses(pre, post, weight, delay, keep)
    sy = sn_synapses()
    sy.m = pre.size
    sy.pre, sy.post, sy.weight, sy.delay = _ptr(pre), _ptr(post), _ptr(w), _ptr(d)
    D = int(max_delay if max_delay is not None else (d.max() if d.size else 1))
    cfg = _config(dtype, D, flags, record_steps, stream)
    h = _P()
    if axonal_delay is None:
        _check(lib().sn_create(C.byref(cfg), C.byref(nr), C.byref(sy), C.byref(h)))
    else:
        ax = _arr(axonal_delay, np.int32)
        if ax.size != nr.n:
            raise ValueError(f"axonal_delay needs {nr.n} values, got {ax.size}")
        keep.append(ax)
        _check(lib().sn_create_axonal(C.byref(cfg), C.byref(nr), C.byref(sy), _ptr(ax), C.byref(h)))
    return Ctx(h, nr.n, cfg.dtype, (nr.n + 31) // 32, "sparse", pre.size)


def sn_create_shard(threshold, leak, reset, refractory, pre, post, weight, delay, first, count, *,
                    dtype=SN_F32, max_delay=None, record_steps=0, stream=None, flags=SN_AUTO) -> Ctx:
    """Shard [first, first + count) of a sparse network (sn_create_shard)."""
    keep = []
    nr = _neurons(threshold, leak, reset, refractory, keep)
    pre, post, w, d = _synapses(pre, post, weight, delay, keep)
    sy = sn_synapses()
    sy.m = pre.size
    sy.pre, sy.post, sy.weight, sy.delay = _ptr(pre), _ptr(post), _ptr(w), _ptr(d)
    D = int(max_delay if max_delay is not None else (d.max() if d.size else 1))
    cfg = _config(dtype, D, flags, record_steps, stream)
    h = _P()
    _check(lib().sn_create_shard(C.byref(cfg), C.byref(nr), C.byref(sy), int(first), int(count), C.byref(h)))
    return Ctx(h, nr.n, cfg.dtype, (nr.n + 31) // 32, "shard", pre.size)


def sn_shard_info(ctx: Ctx):
    """(first, count, steps per exchange) of a shard."""
    f, c, k = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().sn_shard_info(ctx.handle, C.byref(f), C.byref(c), C.byref(k)), ctx)
    return f.value, c.value, k.value


def sn_shard_put_spikes(ctx: Ctx, t0: int, t1: int, bits):
    """The other shards' spike rows of steps [t0, t1): uint32 [t1 - t0, words]
    (numpy, or a CUDA tensor of int32/uint32)."""
    rows = int(t1) - int(t0)
    if hasattr(bits, "data_ptr"):
        if not _is_dev(bits):
            raise ValueError("bits: a torch tensor must be a CUDA tensor")
        _out(bits, rows * ctx.words * 4, "sn_shard_put_spikes (bits)")
        dev = 1
    else:
        bits = np.ascontiguousarray(bits, np.uint32)
        if bits.size < rows * ctx.words:
            raise ValueError(f"bits: need {rows} x {ctx.words} words, got {bits.size}")
        dev = 0
    _check(lib().sn_shard_put_spikes(ctx.handle, int(t0), int(t1), _ptr(bits) if rows else None, dev), ctx)


def from_workload_shard(wl, first, count, *, record_steps=None, stream=None, flags=SN_AUTO) -> Ctx:
    """Shard [first, first + count) of a sparse workload dict, with its inputs."""
    rec = wl["steps"] if record_steps is None else record_steps
    ctx = sn_create_shard(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], wl["pre"], wl["post"],
                          wl["weight"], wl["delay"], first, count, dtype=wl["dtype"],
                          max_delay=wl["max_delay"], record_steps=rec, stream=stream, flags=flags)
    ev = wl["events"]
    if len(ev["step"]):
        sn_set_input(ctx, ev["step"], ev["neuron"], ev["value"])
    po = wl["poisson"]
    if len(po["neuron"]):
        sn_set_poisson(ctx, po["neuron"], po["rate"], po["amplitude"], po["seed"])
    return ctx


def sn_create_dense(threshold, leak, reset, refractory, w, delay=1, *, max_delay=None,
                    flags=SN_AUTO, record_steps=0, stream=None) -> Ctx:
    keep = []
    nr = _neurons(threshold, leak, reset, refractory, keep)
    if w is not None:                  # None: zero weights, set later with sn_set_weights
        w = _arr(w, np.float32)
        if w.size != nr.n * nr.n:
            raise ValueError(f"dense weights: expected {nr.n} x {nr.n} values, got {w.size}")
        keep.append(w)
    cfg = _config(SN_F32, max_delay if max_delay is not None else delay, flags, record_steps, stream)
    h = _P()
    _check(lib().sn_create_dense(C.byref(cfg), C.byref(nr), _ptr(w), int(delay), C.byref(h)))
    return Ctx(h, nr.n, SN_F32, (nr.n + 31) // 32, "dense", nr.n * nr.n)


def sn_create_batch(nets, *, dtype=SN_F32, max_delay, record_steps=0, stream=None) -> Ctx:
    """nets: list of dicts with threshold, leak, reset, refractory, pre, post,
    weight, delay (local indices)."""
    keep = []
    B = len(nets)
    NR = (sn_neurons * B)()
    SY = (sn_synapses * B)()
    total = 0
    words = 0
    for b, d in enumerate(nets):
        nr = _neurons(d["threshold"], d["leak"], d["reset"], d["refractory"], keep)
        NR[b] = nr
        pre, post, w, dl = _synapses(d["pre"], d["post"], d["weight"], d["delay"], keep)
        SY[b].m = pre.size
        SY[b].pre, SY[b].post = _ptr(pre) if pre.size else None, _ptr(post) if post.size else None
        SY[b].weight, SY[b].delay = _ptr(w) if w.size else None, _ptr(dl) if dl.size else None
        total += nr.n
        words += (nr.n + 31) // 32
    cfg = _config(dtype, max_delay, 0, record_steps, stream)
    h = _P()
    _check(lib().sn_create_batch(C.byref(cfg), B, NR, SY, C.byref(h)))
    ctx = Ctx(h, total, cfg.dtype, words, "batch", 0)
    ctx.net_n = [int(np.asarray(d["threshold"]).size) for d in nets]
    return ctx


def sn_create_shared_dense_i8(threshold, leak, reset, refractory, w, trains, *, record_steps=0,
                              stream=None) -> Ctx:
    """Shared dense integer network (weights int8 [n, n], -8..8) driven by
    `trains` input trains."""
    keep = []
    nr = _neurons(threshold, leak, reset, refractory, keep)
    w8 = np.ascontiguousarray(w, np.int8)
    if w8.size != nr.n * nr.n:
        raise ValueError(f"shared weights: expected {nr.n} x {nr.n} values, got {w8.size}")
    cfg = _config(SN_I32, 1, 0, record_steps, stream)
    h = _P()
    _check(lib().sn_create_shared_dense_i8(C.byref(cfg), C.byref(nr), _ptr(w8), int(trains), C.byref(h)))
    ctx = Ctx(h, nr.n * int(trains), SN_I32, nr.n * int(trains) // 32, "shared", nr.n * nr.n)
    ctx.net_n = [nr.n] * int(trains)
    return ctx


def from_shared_workload(wl, *, record_steps=None, stream=None, first_train=0, trains=None) -> Ctx:
    """Shared dense context for a shared_dense_i8 workload.  first_train and
    trains select the trains [first_train, first_train + trains) of the
    workload's family (one shard of it); their Poisson streams keep their
    global train indices."""
    rec = wl["steps"] if record_steps is None else record_steps
    B = wl["batch"] if trains is None else int(trains)
    ctx = sn_create_shared_dense_i8(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"],
                                    wl["dense_w_i8"], B, record_steps=rec, stream=stream)
    po = wl["poisson"]
    if len(po["neuron"]):
        sn_set_poisson_stream(ctx, po["neuron"], po["rate"], po["amplitude"], po["seed"], int(first_train))
    return ctx


def sn_batch_config(ctx: Ctx, warp_max_n: int, ring_smem_bytes: int):
    _check(lib().sn_batch_config(ctx.handle, int(warp_max_n), int(ring_smem_bytes)), ctx)


def sn_autotune(ctx: Ctx, trial_steps: int = 20) -> float:
    ms = C.c_float(0)
    _check(lib().sn_autotune(ctx.handle, int(trial_steps), C.byref(ms)), ctx)
    return ms.value


def sn_set_propagation(ctx: Ctx, mode: int):
    """SN_PUSH or SN_PULL propagation for a sparse network."""
    _check(lib().sn_set_propagation(ctx.handle, int(mode)), ctx)


def sn_get_propagation(ctx: Ctx) -> int:
    m = C.c_int32(0)
    _check(lib().sn_get_propagation(ctx.handle, C.byref(m)), ctx)
    return m.value


def sn_pull_store_info(ctx: Ctx):
    """(format, bytes, entries) of a sparse context's pull store: format 0 (not
    built), SN_PULL_PLAIN or SN_PULL_CODED."""
    f, b, e = C.c_int32(0), C.c_int64(0), C.c_int64(0)
    _check(lib().sn_pull_store_info(ctx.handle, C.byref(f), C.byref(b), C.byref(e)), ctx)
    return f.value, b.value, e.value


def split_batch_raster(bits, net_n):
    """Raster words of a batched context -> list of per-network uint8
    rasters [steps, n_b]."""
    out = []
    w0 = 0
    for n in net_n:
        w = (n + 31) // 32
        out.append(unpack_raster(np.ascontiguousarray(bits[:, w0:w0 + w]), n))
        w0 += w
    return out


def sn_set_input(ctx: Ctx, step, neuron, value):
    s, j = _arr(step, np.int32).reshape(-1), _arr(neuron, np.int32).reshape(-1)
    if s.size != j.size:
        raise ValueError(f"input events: {s.size} steps and {j.size} neurons")
    (v,) = _match("input event values", s.size, _arr(value, np.float32))
    _check(lib().sn_set_input(ctx.handle, s.size, _ptr(s) if s.size else None,
                              _ptr(j) if j.size else None, _ptr(v) if v.size else None), ctx)


def sn_set_poisson(ctx: Ctx, neuron, rate, amplitude, seed):
    j = _arr(neuron, np.int32).reshape(-1)
    r, a = _match("Poisson rates and amplitudes", j.size, _arr(rate, np.float32), _arr(amplitude, np.float32))
    _check(lib().sn_set_poisson(ctx.handle, j.size, _ptr(j) if j.size else None,
                                _ptr(r) if r.size else None, _ptr(a) if a.size else None,
                                int(seed) & (2**64 - 1)), ctx)


def sn_set_poisson_stream(ctx: Ctx, neuron, rate, amplitude, seed, net):
    j = _arr(neuron, np.int32).reshape(-1)
    r, a = _match("Poisson rates and amplitudes", j.size, _arr(rate, np.float32), _arr(amplitude, np.float32))
    _check(lib().sn_set_poisson_stream(ctx.handle, j.size, _ptr(j) if j.size else None,
                                       _ptr(r) if r.size else None, _ptr(a) if a.size else None,
                                       int(seed) & (2**64 - 1), int(net) & (2**64 - 1)), ctx)


def sn_stdp(ctx: Ctx, decay, a_plus, a_minus, wmin, wmax, enable=True):
    _check(lib().sn_stdp(ctx.handle, decay, a_plus, a_minus, wmin, wmax, int(bool(enable))), ctx)


def sn_run(ctx: Ctx, steps: int):
    _check(lib().sn_run(ctx.handle, int(steps)), ctx)


def sn_reset(ctx: Ctx):
    _check(lib().sn_reset(ctx.handle), ctx)


def sn_sync(ctx: Ctx):
    _check(lib().sn_sync(ctx.handle), ctx)


def sn_get_spikes(ctx: Ctx, t0: int, t1: int, out=None):
    """Raster words [(t1 - t0), words] (uint32).  `out` may be a torch CUDA
    tensor of that shape (int32 or uint32 storage) for a device-side copy."""
    if out is None:
        out = np.zeros((t1 - t0, ctx.words), np.uint32)
    _out(out, max(0, t1 - t0) * ctx.words * 4, "sn_get_spikes")
    _check(lib().sn_get_spikes(ctx.handle, int(t0), int(t1), _ptr(out), int(_is_dev(out))), ctx)
    return out


def unpack_raster(bits, n):
    """Raster words -> uint8 [steps, n] (bit j % 32 of word j // 32)."""
    b = np.asarray(bits, dtype=np.uint32)
    u8 = b.view(np.uint8).reshape(b.shape[0], -1)
    return np.unpackbits(u8, axis=1, bitorder="little")[:, :n]


def sn_get_state(ctx: Ctx, v=None, refractory=None):
    vt = np.int32 if ctx.dtype == SN_I32 else np.float32
    if v is None:
        v = np.zeros(ctx.n, vt)
    if refractory is None:
        refractory = np.zeros(ctx.n, np.int32)
    _out(v, ctx.n * 4, "sn_get_state (v)")
    _out(refractory, ctx.n * 4, "sn_get_state (refractory)")
    dev = _is_dev(v)
    _check(lib().sn_get_state(ctx.handle, _ptr(v), _ptr(refractory), int(dev)), ctx)
    return v, refractory


def sn_get_trace(ctx: Ctx, out=None):
    if out is None:
        out = np.zeros(ctx.n, np.float32)
    _out(out, ctx.n * 4, "sn_get_trace")
    _check(lib().sn_get_trace(ctx.handle, _ptr(out), int(_is_dev(out))), ctx)
    return out


def sn_get_weights(ctx: Ctx, out=None):
    if out is None:
        out = np.zeros(ctx.m, np.float32)
    _out(out, ctx.m * 4, "sn_get_weights")
    _check(lib().sn_get_weights(ctx.handle, _ptr(out), int(_is_dev(out))), ctx)
    return out


def sn_set_weights(ctx: Ctx, w):
    """Replace the weights (same layout as sn_get_weights); w is a host array
    or a device tensor."""
    if _is_dev(w):
        _out(w, ctx.m * 4, "sn_set_weights")
        _check(lib().sn_set_weights(ctx.handle, _ptr(w), 1), ctx)
        return
    w = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
    if w.size != ctx.m:
        raise ValueError(f"expected {ctx.m} weights, got {w.size}")
    _check(lib().sn_set_weights(ctx.handle, _ptr(w), 0), ctx)


def sn_get_counters(ctx: Ctx):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().sn_get_counters(ctx.handle, C.byref(a), C.byref(b), C.byref(c)), ctx)
    return a.value, b.value, c.value


def sn_save(ctx: Ctx) -> bytes:
    size = C.c_size_t(0)
    _check(lib().sn_save(ctx.handle, None, C.byref(size)), ctx)
    buf = C.create_string_buffer(size.value)
    _check(lib().sn_save(ctx.handle, buf, C.byref(size)), ctx)
    return buf.raw[:size.value]


def sn_load(ctx: Ctx, blob: bytes):
    _check(lib().sn_load(ctx.handle, blob, len(blob)), ctx)


def _noalloc_arg(t, numel, dtypes, what, device, at_least=False):
    """A CUDA tensor on `device`, contiguous, of one of `dtypes`, holding
    exactly (or, for outputs, at least) `numel` elements: the kernel reads or
    writes that many through the raw pointer."""
    if not _is_dev(t):
        raise ValueError(f"{what}: expected a CUDA tensor, got {type(t).__name__}")
    if t.device != device:
        raise ValueError(f"{what}: on {t.device}, expected {device} (the weights' device)")
    if str(t.dtype).replace("torch.", "") not in dtypes:
        raise ValueError(f"{what}: dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: not contiguous")
    if (t.numel() < numel) if at_least else (t.numel() != numel):
        raise ValueError(f"{what}: {t.numel()} elements, expected {'at least ' if at_least else ''}{numel}")


def sn_run_dense_noalloc(n, delay, steps, w, threshold, leak, reset, refractory, v, r, raster,
                         poisson_threshold=None, poisson_amplitude=None, seed=0, stream=None):
    """Dense run on caller-owned device tensors (torch CUDA tensors, all on
    the current device); the library allocates nothing.  w float32 [n*n];
    threshold, leak, reset, v float32 [n]; refractory, r int32 [n]; raster
    int32 or uint32, at least steps * ceil(n/32) words; poisson_threshold
    int32 or uint32 [n] and poisson_amplitude float32 [n], both or neither.
    Every argument is checked before the C call (ValueError); a non-OK status
    raises SnError."""
    import torch
    n, delay, steps = int(n), int(delay), int(steps)
    if n < 1 or steps < 0:
        raise ValueError(f"n = {n} and steps = {steps}: need n >= 1, steps >= 0")
    if (poisson_threshold is None) != (poisson_amplitude is None):
        raise ValueError("poisson_threshold and poisson_amplitude: give both or neither")
    if not _is_dev(w):
        raise ValueError("w: expected a CUDA tensor")
    device = torch.device("cuda", torch.cuda.current_device())
    words = (n + 31) // 32
    _noalloc_arg(w, n * n, ("float32",), "w", device)
    for t, what in ((threshold, "threshold"), (leak, "leak"), (reset, "reset"), (v, "v")):
        _noalloc_arg(t, n, ("float32",), what, device)
    for t, what in ((refractory, "refractory"), (r, "r")):
        _noalloc_arg(t, n, ("int32",), what, device)
    if steps > 0:
        _noalloc_arg(raster, steps * words, ("int32", "uint32"), "raster", device, at_least=True)
    if poisson_threshold is not None:
        _noalloc_arg(poisson_threshold, n, ("int32", "uint32"), "poisson_threshold", device)
        _noalloc_arg(poisson_amplitude, n, ("float32",), "poisson_amplitude", device)
    a = sn_dense_noalloc_args()
    a.n, a.delay, a.steps = n, delay, steps
    a.w, a.threshold, a.leak, a.reset = _ptr(w), _ptr(threshold), _ptr(leak), _ptr(reset)
    a.refractory = _ptr(refractory)
    a.poisson_threshold, a.poisson_amplitude = _ptr(poisson_threshold), _ptr(poisson_amplitude)
    a.seed = int(seed) & (2**64 - 1)
    a.v, a.r, a.raster = _ptr(v), _ptr(r), _ptr(raster) if steps > 0 else None
    a.cuda_stream = stream
    _check(lib().sn_run_dense_noalloc(C.byref(a)))


def sn_create_ff(sizes, delays, *, threshold, leak, reset, refractory, slope, checkpoint_every,
                 batch, steps, stream=None, recompute=False) -> Ctx:
    """Feedforward context; delays: list of uint8 arrays [n_in, n_out] (host).
    recompute: SN_FF_RECOMPUTE (the backward recomputes the synaptic input)."""
    sz = np.ascontiguousarray(sizes, np.int32)
    ds = [np.ascontiguousarray(d, np.uint8) for d in delays]
    if sz.size != len(ds) + 1:
        raise ValueError(f"{sz.size} layer sizes need {sz.size - 1} delay arrays, got {len(ds)}")
    for l, d in enumerate(ds):
        if d.size != int(sz[l]) * int(sz[l + 1]):
            raise ValueError(f"delays[{l}]: expected {int(sz[l])} x {int(sz[l + 1])} values, got {d.size}")
    ptrs = (C.c_void_p * len(ds))(*[_ptr(d) for d in ds])
    p = sn_ff_params(float(threshold), float(leak), float(reset), int(refractory), float(slope),
                     int(checkpoint_every))
    cfg = _config(SN_F32, 1, SN_FF_RECOMPUTE if recompute else 0, 0, stream)
    h = _P()
    _check(lib().sn_create_ff(C.byref(cfg), len(ds), _ptr(sz), ptrs, C.byref(p), int(batch), int(steps),
                              C.byref(h)))
    ctx = Ctx(h, int(sz[-1]), SN_F32, 0, "ff", 0)
    ctx.sizes, ctx.batch, ctx.steps, ctx.k = [int(x) for x in sz], int(batch), int(steps), int(checkpoint_every)
    return ctx


def sn_ff_set_engine(ctx: Ctx, engine: int):
    _check(lib().sn_ff_set_engine(ctx.handle, int(engine)), ctx)


def _dev(t, numel, dtype, what):
    """A CUDA tensor of `numel` elements of `dtype` ("uint8", "float32"),
    contiguous: the library reads or writes exactly that many."""
    if not _is_dev(t):
        raise ValueError(f"{what}: expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{what}: expected a contiguous {dtype} tensor of {numel} elements, got "
                         f"{t.dtype} with {t.numel()} (contiguous: {t.is_contiguous()})")


def _ff_layers(ctx, tensors, dtype, what):
    L = len(ctx.sizes) - 1
    if len(tensors) != L:
        raise ValueError(f"{what}: expected {L} tensors, got {len(tensors)}")
    for l, t in enumerate(tensors):
        _dev(t, ctx.sizes[l] * ctx.sizes[l + 1], dtype, f"{what}[{l}]")


def sn_ff_forward(ctx: Ctx, input_spikes, weights, counts):
    """input_spikes: CUDA uint8 [steps, batch, n0]; weights: CUDA float32
    tensors [n_in, n_out]; counts: CUDA float32 [batch, n_out] (written)."""
    _dev(input_spikes, ctx.steps * ctx.batch * ctx.sizes[0], "uint8", "input spikes")
    _ff_layers(ctx, weights, "float32", "weights")
    _dev(counts, ctx.batch * ctx.sizes[-1], "float32", "counts")
    ptrs = (C.c_void_p * len(weights))(*[_ptr(w) for w in weights])
    _check(lib().sn_ff_forward(ctx.handle, _ptr(input_spikes), ptrs, _ptr(counts)), ctx)


def sn_backward(ctx: Ctx, grad_counts, grad_weights):
    _dev(grad_counts, ctx.batch * ctx.sizes[-1], "float32", "count gradient")
    _ff_layers(ctx, grad_weights, "float32", "weight gradients")
    ptrs = (C.c_void_p * len(grad_weights))(*[_ptr(g) for g in grad_weights])
    _check(lib().sn_backward(ctx.handle, _ptr(grad_counts), ptrs, 1), ctx)


def sn_ff_get_spikes(ctx: Ctx, layer: int):
    n = ctx.sizes[layer]
    out = np.zeros((ctx.steps, ctx.batch, (n + 31) // 32), np.uint32)
    _check(lib().sn_ff_get_spikes(ctx.handle, int(layer), _ptr(out), 0), ctx)
    b = out.reshape(ctx.steps * ctx.batch, -1)
    return unpack_raster(b, n).reshape(ctx.steps, ctx.batch, n)


def sn_ff_get_checkpoints(ctx: Ctx, layer: int):
    n = ctx.sizes[layer]
    out = np.zeros((ctx.steps // ctx.k, ctx.batch, n), np.float32)
    _check(lib().sn_ff_get_checkpoints(ctx.handle, int(layer), _ptr(out), 0), ctx)
    return out


def sn_selftest_barrier_timeout(stream=None) -> int:
    """Run the failure-detection self-test (a grid barrier that one block
    never reaches); returns the status the kernel latched (SN_ETIMEOUT when
    the wait's bound works)."""
    st = C.c_int32(-1)
    _check(lib().sn_selftest_barrier_timeout(stream, C.byref(st)))
    return st.value


def sn_version() -> str:
    return lib().sn_version().decode()


def sn_destroy(ctx: Ctx):
    if ctx.handle:
        lib().sn_destroy(ctx.handle)
        ctx.handle = None


# ---------------------------------------------------------------------------
# workload helper (marshalling of a workload dict into the calls above)

def from_workload(wl, *, record_steps=None, flags=SN_AUTO, stream=None, w_device=None) -> Ctx:
    """Create a context for a workload dict of paper_2305_02510_gb300.workloads
    and install its inputs (events, Poisson sources, STDP).  A workload whose
    dense weights live on the device (huge_dense) takes them as w_device, a
    device tensor [n, n]."""
    rec = wl["steps"] if record_steps is None else record_steps
    if "dense_w_device" in wl:
        if w_device is None:
            raise ValueError("this workload's weights are a device tensor: pass w_device")
        ctx = sn_create_dense(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], None,
                              wl["dense_delay"], max_delay=wl["max_delay"], flags=flags, record_steps=rec,
                              stream=stream)
        sn_set_weights(ctx, w_device)
    elif "dense_w" in wl:
        ctx = sn_create_dense(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"],
                              wl["dense_w"], wl["dense_delay"], max_delay=wl["max_delay"],
                              flags=flags, record_steps=rec, stream=stream)
    else:
        ctx = sn_create(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], wl["pre"],
                        wl["post"], wl["weight"], wl["delay"], dtype=wl["dtype"],
                        max_delay=wl["max_delay"], flags=flags, record_steps=rec, stream=stream,
                        axonal_delay=wl.get("axonal_delay"))
    ev = wl["events"]
    if len(ev["step"]):
        sn_set_input(ctx, ev["step"], ev["neuron"], ev["value"])
    po = wl["poisson"]
    if len(po["neuron"]):
        sn_set_poisson(ctx, po["neuron"], po["rate"], po["amplitude"], po["seed"])
    if wl.get("stdp"):
        sd = wl["stdp"]
        sn_stdp(ctx, sd["decay"], sd["a_plus"], sd["a_minus"], sd["wmin"], sd["wmax"], True)
    return ctx


def from_batch_workloads(nets, *, record_steps=None, stream=None, first=0) -> Ctx:
    """Batched context for a list of workload dicts (all sparse, same dtype);
    network b of the list is stream first + b of the batch's Poisson input
    (first: the global index of the list's first network when the list is
    one shard of a larger family), whose seed is taken from the first
    network."""
    rec = nets[0]["steps"] if record_steps is None else record_steps
    D = max(int(w["max_delay"]) for w in nets)
    ctx = sn_create_batch(nets, dtype=nets[0]["dtype"], max_delay=D, record_steps=rec, stream=stream)
    off = np.cumsum([0] + [w["n"] for w in nets])
    nj = [np.asarray(w["poisson"]["neuron"], np.int64) + off[b] for b, w in enumerate(nets)]
    if sum(x.size for x in nj):
        sn_set_poisson_stream(ctx, np.concatenate(nj), np.concatenate([w["poisson"]["rate"] for w in nets]),
                              np.concatenate([w["poisson"]["amplitude"] for w in nets]),
                              nets[0]["poisson"]["seed"], int(first))
    evs = [(np.asarray(w["events"]["step"]), np.asarray(w["events"]["neuron"]) + off[b],
            np.asarray(w["events"]["value"])) for b, w in enumerate(nets)]
    if sum(e[0].size for e in evs):
        sn_set_input(ctx, np.concatenate([e[0] for e in evs]), np.concatenate([e[1] for e in evs]),
                     np.concatenate([e[2] for e in evs]))
    return ctx
