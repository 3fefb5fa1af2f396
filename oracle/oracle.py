"""Python front end of the CPU oracle (sn_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The simulator library never imports it.

`run(wl, mode, ...)` takes a workload dict (see paper_2305_02510_gb300.workloads)
and steps the plain C oracle.  Float workloads are rounded to float32 before
either mode sees them, so the fp64 trajectory and the fp32 mirror run the very
same network as the GPU.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "sn_oracle.c")

F64, F32, INT = 0, 1, 2
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sn_oracle.c with gcc (no fused multiply-add, no fast-math)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class OrcNet(C.Structure):
    _fields_ = [
        ("mode", C.c_int32), ("n", C.c_int32), ("max_delay", C.c_int32), ("dense", C.c_int32),
        ("threshold", C.c_void_p), ("leak", C.c_void_p), ("reset", C.c_void_p),
        ("refractory", C.c_void_p),
        ("m", C.c_int64), ("pre", C.c_void_p), ("post", C.c_void_p), ("delay", C.c_void_p),
        ("weight", C.c_void_p),
        ("w_dense", C.c_void_p), ("dense_delay", C.c_int32),
        ("nev", C.c_int64), ("ev_step", C.c_void_p), ("ev_neuron", C.c_void_p),
        ("ev_value", C.c_void_p),
        ("nsrc", C.c_int32), ("src_neuron", C.c_void_p), ("src_rate_u32", C.c_void_p),
        ("src_amp", C.c_void_p), ("seed", C.c_uint64), ("net", C.c_uint64),
        ("stdp", C.c_int32), ("decay", C.c_double), ("a_plus", C.c_double),
        ("a_minus", C.c_double), ("wmin", C.c_double), ("wmax", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_run.argtypes = [C.POINTER(OrcNet), C.c_int64, C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.orc_run.restype = C.c_int
            _lib.orc_poisson_u32.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32]
            _lib.orc_poisson_u32.restype = C.c_uint32
            _lib.orc_splitmix64.argtypes = [C.c_uint64]
            _lib.orc_splitmix64.restype = C.c_uint64
            _lib.orc_set_threads.argtypes = [C.c_int]
            _lib.orc_set_threads.restype = C.c_int
    return _lib


def set_threads(k: int) -> int:
    """Threads for the per-neuron loop of each oracle step (1 by default).
    Each neuron's step depends only on earlier steps and its own state, so
    the results do not depend on k."""
    return int(lib().orc_set_threads(int(k)))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & (2**64 - 1))))


def poisson_u32(seed: int, net: int, t: int, j: int) -> int:
    return int(lib().orc_poisson_u32(seed, net, t, j))


def rate_to_u32(rate) -> np.ndarray:
    """Firing probability per step as a 32-bit threshold: floor(rate * 2^32),
    clamped to [0, 2^32 - 1]; a source fires when its uniform is below it."""
    r = np.floor(np.asarray(rate, np.float64) * 4294967296.0)
    return np.clip(r, 0, 4294967295).astype(np.uint32)


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


def canon(wl, mode):
    """Float workloads rounded to float32 (the precision the library stores);
    integer workloads unchanged."""
    f = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if wl["dtype"] == "f32" \
        else (lambda a: np.asarray(a, np.float64))
    return f


class State:
    """Oracle state between calls: V, refractory countdown, last-D spike rows,
    STDP trace and (possibly plastic) weights."""

    def __init__(self, wl):
        n, D = wl["n"], wl["max_delay"]
        f = canon(wl, None)
        self.t = 0
        self.v = f(wl["reset"]).copy()
        self.r = np.zeros(n, np.int32)
        self.hist = np.zeros((D, n), np.uint8)
        self.trace = np.zeros(n, np.float64)
        if "dense_w" in wl:
            self.w = f(wl["dense_w"]).reshape(-1).copy()
        elif "dense_w_i8" in wl:
            self.w = np.asarray(wl["dense_w_i8"], np.float64).reshape(-1).copy()
        else:
            self.w = f(wl["weight"]).copy()

    def copy(self):
        s = State.__new__(State)
        s.t = self.t
        for k in ("v", "r", "hist", "trace", "w"):
            setattr(s, k, getattr(self, k).copy())
        return s


def run(wl, mode: int, steps: int, state: State | None = None, record_v: bool = False,
        net_index: int = 0, poisson_seed: int | None = None):
    """Advance the oracle `steps` timesteps from `state` (fresh if None).

    Returns (state, raster[steps, n] uint8, vtrace[steps, n] or None); with
    record_v the state compared with the threshold in each step is kept in
    state.ctrace.
    """
    L = lib()
    n, D = wl["n"], wl["max_delay"]
    st = State(wl) if state is None else state
    f = canon(wl, mode)
    th, lk, rs = f(wl["threshold"]), f(wl["leak"]), f(wl["reset"])
    rf = np.ascontiguousarray(wl["refractory"], np.int32)
    keep = [th, lk, rs, rf]
    net = OrcNet()
    net.mode, net.n, net.max_delay = mode, n, D
    net.threshold, net.leak, net.reset, net.refractory = _p(th), _p(lk), _p(rs), _p(rf)
    dense = "dense_w" in wl or "dense_w_i8" in wl
    net.dense = int(dense)
    if dense:
        net.w_dense = _p(st.w)
        net.dense_delay = int(wl["dense_delay"])
    else:
        pre = np.ascontiguousarray(wl["pre"], np.int32)
        post = np.ascontiguousarray(wl["post"], np.int32)
        dl = np.ascontiguousarray(wl["delay"], np.int32)
        if wl.get("axonal_delay") is not None:
            # Section 2.2: the axonal delay is a neuron parameter; a spike
            # crosses the pre-neuron's axon, then the synapse
            dl = np.ascontiguousarray(dl + np.asarray(wl["axonal_delay"], np.int32)[pre], np.int32)
        keep += [pre, post, dl]
        net.m = pre.size
        net.pre, net.post, net.delay, net.weight = _p(pre), _p(post), _p(dl), _p(st.w)
    ev = wl["events"]
    es = np.ascontiguousarray(ev["step"], np.int32)
    en = np.ascontiguousarray(ev["neuron"], np.int32)
    evv = f(ev["value"])
    keep += [es, en, evv]
    net.nev, net.ev_step, net.ev_neuron, net.ev_value = es.size, _p(es), _p(en), _p(evv)
    po = wl["poisson"]
    sn = np.ascontiguousarray(po["neuron"], np.int32)
    # sn_set_poisson takes the rate as a float32: threshold of the rounded rate
    su = rate_to_u32(np.asarray(po["rate"], np.float32).astype(np.float64))
    sa = f(po["amplitude"])
    keep += [sn, su, sa]
    net.nsrc, net.src_neuron, net.src_rate_u32, net.src_amp = sn.size, _p(sn), _p(su), _p(sa)
    net.seed = int(po["seed"] if poisson_seed is None else poisson_seed) & (2**64 - 1)
    net.net = int(net_index)
    sd = wl.get("stdp")
    if sd:
        net.stdp = 1
        if mode == F32:
            q = lambda x: float(np.float32(x))
        else:
            q = float
        net.decay, net.a_plus, net.a_minus = q(sd["decay"]), q(sd["a_plus"]), q(sd["a_minus"])
        net.wmin, net.wmax = q(sd["wmin"]), q(sd["wmax"])
    raster = np.zeros((steps, n), np.uint8)
    vtr = np.zeros((steps, n), np.float64) if record_v else None
    ctr = np.zeros((steps, n), np.float64) if record_v else None
    rc = L.orc_run(C.byref(net), st.t, steps, _p(st.v), _p(st.r), _p(st.hist),
                   _p(st.trace), _p(raster), _p(vtr) if vtr is not None else None,
                   _p(ctr) if ctr is not None else None)
    st.ctrace = ctr
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")
    st.t += steps
    del keep
    return st, raster, vtr


def state_from(wl, t, v, r, raster_rows, trace=None, w=None):
    """Oracle state at absolute step t built from outside values: V and the
    refractory countdown after step t-1, and the spike rows of steps
    t-D .. t-1 (rows of [D, n], zero for steps before 0)."""
    st = State(wl)
    st.t = int(t)
    st.v = np.asarray(v, np.float64).copy()
    st.r = np.asarray(r, np.int32).copy()
    st.hist = np.ascontiguousarray(raster_rows, np.uint8).copy()
    if trace is not None:
        st.trace = np.asarray(trace, np.float64).copy()
    if w is not None:
        st.w = np.asarray(w, np.float64).reshape(-1).copy()
    return st
