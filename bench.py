#!/usr/bin/env python
"""Throughput benchmark of the spiking-network simulator on one GB300.

One benchmark step = one full simulation of the large sparse network
(N = 100,000 LIF neurons, 100 synapses each = 1e7 synapses, delays 1..16,
float32 state, Poisson input into 1% of the neurons) for 1000 timesteps, from
the initial state.  Headline metric: synaptic events per second (one event =
one spike delivered along one synapse), with timesteps per second beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank simulates its own replica of the network with its own
input stream (the single network is not sharded: replicas only, weak scaling).
The reference arm (--impl reference) times the CPU oracle on bounded samples
of the same workload on this host; only rank 0 runs it.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "synaptic events/s & timesteps/s on 1 GB300 (batched vs plain); BPTT step ms"
UNIT = "synaptic events/s"
TIMESTEPS = 1000
# per-neuron state bytes touched once per timestep by the update phase:
# V and r read+write (16), threshold/leak/reset/refractory/Poisson rate and
# amplitude read (24), pending-input slot read and clear (16)
STATE_BYTES = 56
# the pull kernel touches the same state without the pending-input slot
STATE_BYTES_PULL = 40
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch per
# kernel, as measured by ncu, with a hash of the sources that kernel is built
# from when it was measured; a figure whose sources changed since is stale and
# not reported (bench.py --record-traffic writes this file from an ncu CSV)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
CSRC = os.path.join(ROOT, "paper_2305_02510_gb300", "csrc")
KERNEL_SOURCES = {
    "sparse_pull_kernel": ["sn_pull.cu", "sn_device.cuh", "sn_internal.h"],
    "sparse_reg_kernel": ["sn_kernels.cu", "sn_device.cuh", "sn_internal.h"],
    "dense_kernel": ["sn_kernels.cu", "sn_device.cuh", "sn_internal.h"],
    "batch_kernel": ["sn_batch.cu", "sn_device.cuh", "sn_internal.h"],
    "shared_kernel": ["sn_shared.cu", "sn_tc.cuh", "sn_device.cuh", "sn_internal.h"],
}


def kernel_source_hash(kernel):
    """sha256 (first 16 hex digits) of the source files a kernel is built from."""
    import hashlib
    base = kernel.split("<")[0]
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[base]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from TRAFFIC_FILE, or
    (None, reason) when none was recorded or the kernel's sources changed."""
    try:
        with open(TRAFFIC_FILE) as f:
            rows = [ln.split("\t") for ln in f.read().splitlines() if ln and not ln.startswith("#")]
    except OSError:
        return None, "no ncu traffic recorded"
    for r in rows:
        if len(r) >= 5 and r[0] == kernel and r[1] == workload:
            if r[2] != kernel_source_hash(kernel):
                return None, "kernel changed since its ncu capture"
            return float(r[3]), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, commit {r[4]}"
    return None, "no ncu traffic recorded for this kernel and workload"


def record_traffic(csv_path, kernel, workload, launches_per_unit=1):
    """Add (or replace) the TRAFFIC_FILE line of `kernel` on `workload` from an
    ncu --csv capture with dram__bytes_read.sum and dram__bytes_write.sum: the
    mean over the captured launches of that kernel, in bytes."""
    import csv
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    per = {}
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        if kernel.split("<")[0] + "<" not in row.get("Kernel Name", ""):
            continue
        if row.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        v = float(row["Metric Value"].replace(",", "")) * unit.get(row.get("Metric Unit", "byte"), 1)
        per.setdefault(row["ID"], 0.0)
        per[row["ID"]] += v
    if not per:
        raise SystemExit(f"no dram__bytes rows for {kernel} in {csv_path}")
    value = launches_per_unit * sum(per.values()) / len(per)
    commit = subprocess.run(["git", "-C", ROOT, "rev-parse", "--short", "HEAD"], capture_output=True,
                            text=True).stdout.strip() or "unknown"
    keep = []
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            keep = [ln for ln in f.read().splitlines()
                    if ln and not ln.startswith("#") and ln.split("\t")[:2] != [kernel, workload]]
    with open(TRAFFIC_FILE, "w") as f:
        f.write("# kernel\tworkload\tsource sha256 (16)\tDRAM bytes per launch\tcommit measured\n")
        for ln in keep + [f"{kernel}\t{workload}\t{kernel_source_hash(kernel)}\t{value:.6g}\t{commit}"]:
            f.write(ln + "\n")
    print(f"{kernel} on {workload}: {value:.4g} B per launch ({len(per)} launches)")


def replica_seed(seed, rank):
    """Poisson seed of replica `rank`: every rank simulates its own copy of the
    network with its own input stream."""
    return int(seed) + 7919 * int(rank)


def combine_ranks(ms, events, e2e_s, e2e_events, world, device):
    """Whole-job figures over the ranks: the slowest rank's time (max) and the
    total work (sum).  With world == 1 the local figures."""
    if world <= 1:
        return ms, events, e2e_s, e2e_events
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, events, e2e_s, e2e_events], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(mx[2]), float(sm[3])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons.  The
    sampler starts before the warm-up so that it is running when the timed
    region begins; the summary keeps the samples whose timestamps fall inside
    the marked region (or, for a region shorter than the sampling interval,
    the samples nearest to it)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.t0 = self.t1 = None
        self.rows = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.p is None:
            return
        time.sleep(0.1)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        import datetime
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            self.rows.append((ts, f[1:]))

    def summary(self):
        if not self.rows or self.t0 is None or self.t1 is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = [r for ts, r in self.rows if self.t0 <= ts <= self.t1]
        window = "timed region"
        if not inside:
            mid = 0.5 * (self.t0 + self.t1)
            near = sorted(self.rows, key=lambda x: abs(x[0] - mid))[:2]
            inside = [r for _, r in near]
            window = "nearest to a timed region shorter than the 50 ms sampling interval"
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "window": window}


def algorithmic_bytes(n, timesteps, spikes, events):
    """Bytes the sparse path must move per launch: per spike its CSR row
    bounds (16 B); per event its packed synapse (8 B) and its accumulate into
    the pending-input ring (8 B); per neuron and timestep the update phase's
    state traffic and its raster bit."""
    return spikes * 16 + events * 16 + timesteps * n * STATE_BYTES + timesteps * n / 8


def algorithmic_bytes_pull(n, m, timesteps):
    """Bytes pull propagation must move per launch: every timestep each
    neuron's incoming synapses (8 B each, packed pre | delay and weight) and
    the update phase's state traffic and raster bit.  The spike-history rows
    each block copies into shared memory are not counted (L2 reads of a few
    MB per step)."""
    return timesteps * (m * 8 + n * STATE_BYTES_PULL + n / 8)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(wl, warm=40, timed=60):
    """The CPU oracle as it stands on a bounded sample of the workload: `warm`
    untimed timesteps from the initial state (past the start-up transient),
    then `timed` timesteps timed single-threaded and again on every host core
    (the per-neuron loop split over threads; identical results).  Returns a
    dict per thread count: events/s, timesteps/s, threads, sample text."""
    from oracle import oracle as O
    deg = np.bincount(np.asarray(wl["pre"]), minlength=wl["n"]).astype(np.int64)
    cores = host_cores()
    O.set_threads(cores)
    try:
        base, _, _ = O.run(wl, O.F32, warm)
        out = {}
        for k in (1, cores):
            O.set_threads(k)
            t0 = time.perf_counter()
            st, raster, _ = O.run(wl, O.F32, timed, state=base.copy())
            dt = time.perf_counter() - t0
            ev = int((raster.astype(np.int64) * deg[None, :]).sum())
            out[k] = {"value": ev / dt, "timesteps_per_s": timed / dt, "cores": k,
                      "sample": f"timesteps {warm}..{warm + timed - 1} of {wl['name']} (N={wl['n']}, "
                                f"M={len(wl['pre'])}), C oracle (float32 mirror) on {k} thread(s) "
                                f"of {cores} host cores"}
    finally:
        O.set_threads(1)
    return out


def event_bytes(n, timesteps, spikes, events, state_bytes=STATE_BYTES):
    """The method's own bytes per launch, proportional to its events: per
    spike its CSR row bounds (16 B), per event its synapse (8 B) and one
    accumulate into the target's pending input (8 B), per neuron and timestep
    the update's state traffic and its raster bit.  This is the event-driven
    work whichever propagation form runs."""
    return spikes * 16 + events * 16 + timesteps * n * (state_bytes + 1 / 8)


def timed_runs(S, torch, stream, flush, ctx, steps, reps, warm=1):
    """Device time of `reps` runs of `steps` timesteps from the initial state,
    L2 flushed before each; returns (mean ms, spikes, events) per run."""
    out = []
    for k in range(warm + reps):
        S.sn_reset(ctx)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.sn_run(ctx, steps)
        b.record(stream)
        S.sn_sync(ctx)
        _, spk, ev = S.sn_get_counters(ctx)
        if k >= warm:
            out.append((a.elapsed_time(b), spk, ev))
    return (sum(x[0] for x in out) / reps, sum(x[1] for x in out) / reps, sum(x[2] for x in out) / reps)


def extras(S, W, torch, stream, flush):
    """Dense all-to-all network (16384 neurons, 1000 timesteps) without and
    with STDP; 4096 batched networks (500 timesteps) in one launch against
    the plain path (one single-network context and launch per network)."""
    peak, src = peaks()
    res = {}
    # dense, delay 1
    for stdp in (False, True):
        wl = W.large_dense(stdp=stdp, steps=1000)
        ctx = S.from_workload(wl, record_steps=1000, stream=stream.cuda_stream)
        ms, spk, ev = timed_runs(S, torch, stream, flush, ctx, 1000, 2)
        n = wl["n"]
        # per spike: its weight row (4n B); per neuron and step: the update's
        # state traffic
        abytes = spk * 4 * n + 1000 * n * STATE_BYTES
        sector_bytes = None
        if stdp:
            # spiking rows written back; spiking columns read+written in every
            # other row (4 B each way per element)
            col = spk * (n - spk / 1000)
            abytes += spk * 4 * n + col * 8
            # the same at the memory's granularity: a column element is alone in
            # its 32-byte sector at this density, so reading it moves 32 B
            # (writes of unchanged weights are skipped, so none are counted)
            sector_bytes = abytes - col * 8 + col * 32
        line_ = {
            "workload": wl["name"], "neurons": n, "timesteps": 1000, "ms": ms,
            "synaptic_events_per_s": ev / (ms / 1e3), "timesteps_per_s": 1000 / (ms / 1e3),
            "spikes_per_timestep": spk / 1000,
            "roofline": {"bound": "hbm", "achieved": abytes / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": abytes / (ms / 1e3) / 1e9 / peak, "peak_source": src,
                         "kernel": "dense_kernel<1,true,false>" if stdp else "dense_kernel<1,false,true>"}}
        if sector_bytes is not None:
            line_["roofline"]["frac_sector_reads"] = sector_bytes / (ms / 1e3) / 1e9 / peak
            line_["roofline"]["sector_note"] = ("column pass counted at 32 B per element read (one sector "
                                                "each), unchanged weights not written")
        res["dense_stdp" if stdp else "dense"] = line_
        del ctx
    res["dense_stdp"]["stdp_overhead"] = res["dense_stdp"]["ms"] / res["dense"]["ms"]
    # batched networks against the plain per-network path
    nets = W.batched_nets(count=4096, steps=500)
    ctx = S.from_batch_workloads(nets, record_steps=500, stream=stream.cuda_stream)
    S.sn_autotune(ctx, 10)
    ms, spk, ev = timed_runs(S, torch, stream, flush, ctx, 500, 3)
    del ctx
    plain = []
    for b, wl in enumerate(nets):
        c = S.sn_create(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], wl["pre"], wl["post"],
                        wl["weight"], wl["delay"], max_delay=8, record_steps=1, stream=stream.cuda_stream)
        po = wl["poisson"]
        S.sn_set_poisson_stream(c, po["neuron"], po["rate"], po["amplitude"], po["seed"], b)
        plain.append(c)
    for c in plain[:64]:
        S.sn_run(c, 500)
    torch.cuda.synchronize()
    for c in plain:
        S.sn_reset(c)
    flush.zero_()
    a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for c in plain:
        S.sn_run(c, 500)
    b2.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b2)
    plain_ev = sum(S.sn_get_counters(c)[2] for c in plain)
    del plain
    res["tiny"] = tiny_extra(S, W, torch, stream, flush)
    res["paper_grid"] = paper_grid_extra(S, W, torch, stream, flush)
    res["huge_dense"] = huge_dense_extra(S, W, torch, stream, flush)
    res["bptt"] = bptt_extra(S, W, torch, stream)
    res["shared_dense"] = shared_extra(S, W, torch, stream, flush)
    peak, src = peaks()
    nsum = int(sum(w["n"] for w in nets))
    # per neuron and step the update's state traffic; per spike its CSR row
    # bounds; per event its packed synapse (6 B) and its accumulate (8 B)
    bbytes = 500 * nsum * STATE_BYTES + spk * 16 + ev * 14
    res["batched"] = {
        "workload": "4096 networks, N log-uniform [64, 4096], p U(0.01, 0.2), delays 1..8",
        "roofline": {"bound": "hbm", "achieved": bbytes / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bbytes / (ms / 1e3) / 1e9 / peak, "peak_source": src, "kernel": "batch_kernel<SN_F32>",
                     "note": "per-network timestep latency bounds this kernel (quiet networks, one executor each)"},
        "networks": len(nets), "neurons": nsum,
        "synapses": int(sum(len(w["pre"]) for w in nets)), "timesteps": 500, "ms": ms,
        "synaptic_events_per_s": ev / (ms / 1e3), "network_timesteps_per_s": len(nets) * 500 / (ms / 1e3),
        "plain_ms": plain_ms, "plain_synaptic_events_per_s": plain_ev / (plain_ms / 1e3),
        "speedup_vs_plain": plain_ms / ms, "launches": 1, "plain_launches": len(nets)}
    return res


class _Spike:
    """Surrogate spike for the plain-torch comparison path of the BPTT
    measurement (fast sigmoid, slope 10)."""

    @staticmethod
    def make(torch):
        class F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, x, slope):
                ctx.save_for_backward(x)
                ctx.slope = slope
                return (x > 0).to(x.dtype)

            @staticmethod
            def backward(ctx, g):
                (x,) = ctx.saved_tensors
                return g / (1.0 + ctx.slope * x.abs()) ** 2, None
        return F


def plain_torch_bptt_step(torch, task, x, ws, masks, labels, spike):
    """The same training step written as plain torch on the GPU: unrolled over
    the steps, one masked matmul per delay and layer, autograd backward."""
    T, B = task["steps"], task["batch"]
    th, lk, rs = task["threshold"], task["leak"], task["reset"]
    sizes = task["sizes"]
    V = [torch.full((B, n), rs, device=x.device) for n in sizes[1:]]
    hist = [[x[t].float() for t in range(T)]] + [[None] * T for _ in sizes[1:]]
    counts = torch.zeros((B, sizes[-1]), device=x.device)
    wd = [[w * m for m in ms] for w, ms in zip(ws, masks)]
    for t in range(T):
        for l in range(len(ws)):
            I = torch.zeros((B, sizes[l + 1]), device=x.device)
            for d in range(1, len(masks[l]) + 1):
                if t - d >= 0:
                    I = I + hist[l][t - d] @ wd[l][d - 1]
            dv = V[l] - rs
            far = dv.abs().detach() > lk
            u = torch.where(far, V[l] - lk * torch.sign(dv.detach()), torch.full_like(V[l], rs)) + I
            sp = spike.apply(u - th, task["slope"])
            V[l] = u * (1 - sp.detach()) + rs * sp.detach()
            hist[l + 1][t] = sp
        counts = counts + hist[-1][t]
    loss = torch.nn.functional.cross_entropy(counts, labels)
    loss.backward()
    return loss


def bptt_extra(S, W, torch, stream):
    """Training step (forward + backward) of the 700-1024-1024-20 network,
    batch 128, 100 steps, through SNNFunction, against the same step in plain
    torch on the same GPU."""
    from paper_2305_02510_gb300 import bptt
    task = W.bptt_task()
    dev = torch.device("cuda")
    net = bptt.FFNet.from_task(task)
    x = torch.tensor(task["input"], device=dev)
    labels = torch.tensor(task["labels"], device=dev)
    ws = [torch.tensor(w, device=dev, requires_grad=True) for w in task["w"]]

    def ours():
        for w in ws:
            w.grad = None
        counts = bptt.SNNFunction.apply(net, x, *ws)
        torch.nn.functional.cross_entropy(counts, labels).backward()

    def timed(fn, warm, reps):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms = timed(ours, 3, 10)
    net_simt = bptt.FFNet.from_task(task, engine="simt")

    def ours_simt():
        for w in ws:
            w.grad = None
        counts = bptt.SNNFunction.apply(net_simt, x, *ws)
        torch.nn.functional.cross_entropy(counts, labels).backward()

    simt_ms = timed(ours_simt, 3, 10)
    masks = [[torch.tensor(task["delay"][l] == d, device=dev, dtype=torch.float32) for d in range(1, 5)]
             for l in range(len(ws))]
    spike = _Spike.make(torch)
    wp = [torch.tensor(w, device=dev, requires_grad=True) for w in task["w"]]

    def plain():
        for w in wp:
            w.grad = None
        plain_torch_bptt_step(torch, task, x, wp, masks, labels, spike)

    plain_ms = timed(plain, 1, 3)
    sizes = task["sizes"]
    syn = sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    # tensor-core work of one step as executed (padded tiles: K to 64, N to 128
    # for the forward and spike gradient, M to 128 for the weight gradient):
    # forward 12 passes (its synaptic input is kept for the backward), spike
    # gradient 12 passes (layers above the first), weight gradient 8 passes
    rows = task["steps"] * task["batch"]
    up = lambda x, m: (x + m - 1) // m * m
    flop = 0
    for l in range(1, len(sizes)):
        nin, nout = sizes[l - 1], sizes[l]
        flop += 12 * 2 * rows * up(nin, 64) * up(nout, 128)
        if l > 1:
            flop += 12 * 2 * rows * up(nout, 64) * up(nin, 128)
        flop += 8 * 2 * up(nin, 128) * up(nout, 128) * up(rows, 64)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16, src = float(json.load(f)["bf16_tflops"]), "measured bf16 burst"
    except Exception:
        bf16, src = 1900.0, "fallback bf16"
    # the method's own work of one training step, dense-equivalent: forward
    # synaptic input 2*B*T*sum(n_in*n_out); spike gradients of the layers above
    # the first 2*B*T*sum_{l>1}(n_in*n_out); weight gradients as the forward
    alg = 2 * rows * syn + 2 * rows * sum(a * b for a, b in zip(sizes[1:-1], sizes[2:])) + 2 * rows * syn
    return {"workload": "700-1024-1024-20 LIF, per-synapse delays 1..4, batch 128, 100 steps, "
                        "checkpoint every 10", "synapses": syn, "ms_per_training_step": ms,
            "roofline": {"bound": "tensor", "achieved": alg / (ms / 1e3) / 1e12, "peak": bf16, "unit": "TFLOP/s",
                         "frac": alg / (ms / 1e3) / 1e12 / bf16, "peak_source": src,
                         "kernel": "ff_tc_fwd_kernel + ff_tc_kernel (whole step's work over the step time)",
                         "algorithmic_flop_per_step": alg,
                         "executed_tensor_flop_per_step": flop,
                         "executed_frac": flop / (ms / 1e3) / 1e12 / bf16,
                         "note": "executed work counts every delay pass, weight part and padded tile"},
            "engine": "tcgen05 BF16 contractions (forward: exact three-part weight split, block-wise FP32 sums)",
            "simt_engine_ms_per_training_step": simt_ms,
            "plain_torch_ms_per_training_step": plain_ms, "speedup_vs_plain_torch": plain_ms / ms}


def shared_extra(S, W, torch, stream, flush):
    """8192-neuron integer network shared by 256 Poisson input trains, 500
    steps: one persistent launch whose per-step propagation is an exact FP8
    tcgen05 GEMM, against the plain path (the single-network dense simulator
    run once per train, same network, same input streams)."""
    wl = W.shared_dense_i8()
    n, B, T = wl["n"], wl["batch"], 500
    ctx = S.from_shared_workload(wl, record_steps=T, stream=stream.cuda_stream)
    ms, spk, ev = timed_runs(S, torch, stream, flush, ctx, T, 3)
    del ctx
    ops = 2.0 * B * n * n * T
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        peak, src = 2.0 * bf16, "measured bf16 burst x 2 (nominal fp8/bf16 ratio)"
    except Exception:
        peak, src = 2.0 * 1900.0, "fallback bf16 x 2"
    po = wl["poisson"]
    plain = S.sn_create_dense(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"],
                              wl["dense_w_i8"].astype(np.float32), 1, record_steps=1, stream=stream.cuda_stream)
    S.sn_set_poisson_stream(plain, po["neuron"], po["rate"], po["amplitude"], po["seed"], 0)
    S.sn_run(plain, T)
    torch.cuda.synchronize()
    total, pev = 0.0, 0
    for b in range(B):
        S.sn_set_poisson_stream(plain, po["neuron"], po["rate"], po["amplitude"], po["seed"], b)
        S.sn_reset(plain)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.sn_run(plain, T)
        c.record(stream)
        S.sn_sync(plain)
        total += a.elapsed_time(c)
        pev += S.sn_get_counters(plain)[2]
    return {"workload": "8192-neuron int8-weight network (-8..8), 256 Poisson trains, 500 steps",
            "ms": ms, "synaptic_events_per_s": ev / (ms / 1e3), "spikes_per_train_step": spk / (B * T),
            "roofline": {"bound": "tensor", "achieved": ops / (ms / 1e3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": ops / (ms / 1e3) / 1e12 / peak, "peak_source": src,
                         "kernel": "shared_kernel (tcgen05.mma kind::f8f6f4)"},
            "plain_ms": total, "plain_synaptic_events_per_s": pev / (total / 1e3),
            "speedup_vs_plain": total / ms, "launches": 1, "plain_launches": B}


# Table 2 of the paper: seconds for 1000 timesteps on its benchmark networks,
# by simulator, N in (100, 1000, 10000) x p in (.25, .5, .75, 1); None = ">1h".
# MAT ran on a desktop CPU, ABM and BindsNET on an unnamed GPU (Section 3).
PAPER_TABLE2 = {
    "mat": [[0.04, 0.04, 0.05, 0.05], [0.36, 0.52, 0.68, 0.80], [30.37, 40.34, 55.38, 71.62]],
    "abm": [[1.10, 1.16, 1.18, 1.26], [4.11, 5.59, 7.22, 9.08], [166.72, 325.30, 488.83, 641.36]],
    "nest": [[0.41, 0.65, 0.91, 1.23], [28.05, 61.42, 81.54, 112.82], [3242.83, None, None, None]],
    "brian2": [[6.63, 12.43, 18.36, 24.23], [612.43, 1249.31, 1892.19, 2529.77], [None, None, None, None]],
    "bindsnet": [[2.44, 2.34, 2.46, 2.38], [3.45, 3.67, 4.19, 4.64], [63.73, 117.78, 181.04, 230.07]],
}
GRID_N = (100, 1000, 10000)
GRID_P = (0.25, 0.5, 0.75, 1.0)


def tiny_extra(S, W, torch, stream, flush):
    """The tiny network (100 neurons, p = 0.05, delays 1..4, Poisson input
    into 10 neurons), float and integer copies, 1000 timesteps in one launch:
    a latency-bound run reported in timesteps/s."""
    out = {}
    for integer in (False, True):
        wl = W.tiny(integer=integer, steps=1000)
        ctx = S.from_workload(wl, record_steps=1000, stream=stream.cuda_stream)
        S.sn_autotune(ctx, 1000)
        prop = "pull" if S.sn_get_propagation(ctx) == S.SN_PULL else "push"
        ms, spk, ev = timed_runs(S, torch, stream, flush, ctx, 1000, 3)
        out["int" if integer else "float"] = {
            "workload": wl["name"], "ms": ms, "timesteps_per_s": 1000 / (ms / 1e3),
            "synaptic_events_per_s": ev / (ms / 1e3), "spikes_per_timestep": spk / 1000, "propagation": prop}
        del ctx
    return out


def huge_dense_extra(S, W, torch, stream, flush, n=100_000, steps=1000):
    """The paper's 100,000-neuron all-to-all network (Section 4: about five
    minutes in its matrix mode, step count not stated): 40 GB of float32
    weights drawn on the device, 1000 timesteps."""
    peak, src = peaks()
    wl = W.huge_dense(n=n, steps=steps)
    w = W.dense_weights_on_device(wl, torch)
    ctx = S.from_workload(wl, record_steps=steps, stream=stream.cuda_stream, w_device=w)
    del w
    torch.cuda.empty_cache()
    ms, spk, ev = timed_runs(S, torch, stream, flush, ctx, steps, 2)
    del ctx
    torch.cuda.empty_cache()
    abytes = spk * 4 * n + steps * n * STATE_BYTES
    return {"workload": wl["name"] + " (all-to-all, 4e10 B of weights)", "neurons": n, "timesteps": steps,
            "ms": ms, "synaptic_events_per_s": ev / (ms / 1e3), "timesteps_per_s": steps / (ms / 1e3),
            "spikes_per_timestep": spk / steps, "paper": "about 5 minutes, step count not stated (Section 4)",
            "roofline": {"bound": "hbm", "achieved": abytes / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": abytes / (ms / 1e3) / 1e9 / peak, "peak_source": src,
                         "kernel": "dense_kernel<8,false,true>"}}


def paper_grid_extra(S, W, torch, stream, flush):
    """The paper's benchmark grid (Section 3): each network simulated for
    1000 timesteps through the dense path and through the sparse path (push or
    pull, whichever sn_autotune picks), beside the paper's Table 2 times."""
    out = []
    for a, n in enumerate(GRID_N):
        for b, p in enumerate(GRID_P):
            wl = W.paper_grid(n, p, steps=1000)
            m = int(len(wl["pre"]))
            row = {"n": n, "p": p, "synapses": m}
            w = np.zeros((n, n), np.float32)
            w[wl["pre"], wl["post"]] = 1.0
            ctx = S.sn_create_dense(wl["threshold"], wl["leak"], wl["reset"], wl["refractory"], w, 1,
                                    max_delay=1, record_steps=1000, stream=stream.cuda_stream)
            del w
            ev = wl["events"]
            S.sn_set_input(ctx, ev["step"], ev["neuron"], ev["value"])
            ms, spk, _ = timed_runs(S, torch, stream, flush, ctx, 1000, 2)
            row["dense_ms"] = ms
            del ctx
            ctx = S.from_workload(wl, record_steps=1000, stream=stream.cuda_stream)
            S.sn_autotune(ctx, 1000)
            prop = "pull" if S.sn_get_propagation(ctx) == S.SN_PULL else "push"
            ms2, spk2, evs = timed_runs(S, torch, stream, flush, ctx, 1000, 2)
            del ctx
            row["sparse_ms"], row["sparse_propagation"] = ms2, prop
            assert spk2 == spk, "dense and sparse paths disagree on the spike count"
            # events along existing synapses (the dense path also visits the zeros)
            row["synaptic_events"] = evs
            best = min(ms, ms2)
            row["best_s_per_1000_steps"] = best / 1e3
            row["synaptic_events_per_s"] = evs / (best / 1e3)
            for k, tab in PAPER_TABLE2.items():
                row[f"paper_{k}_s"] = tab[a][b]
            row["speedup_vs_paper_mat"] = PAPER_TABLE2["mat"][a][b] / (best / 1e3)
            out.append(row)
    return {"workload": "paper benchmark grid (Section 3): Bernoulli(p) digraphs, unit weights and delays, "
                        "3 inputs spiked every 10 steps, 1000 timesteps; paper times are Table 2 "
                        "(desktop CPU / unnamed GPU)", "points": out}


def run_reference(args, wl, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    deg = np.bincount(np.asarray(wl["pre"]), minlength=wl["n"]).astype(np.int64)
    cores = host_cores()
    O.set_threads(cores)
    base, _, _ = O.run(wl, O.F32, 40)
    per = 16
    times, evs = [], []
    for k in range(args.warmup + args.steps):
        st = base.copy()
        t0 = time.perf_counter()
        st, raster, _ = O.run(wl, O.F32, per, state=st)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            evs.append(int((raster.astype(np.int64) * deg[None, :]).sum()))
    O.set_threads(1)
    value = sum(evs) / sum(times)
    sample = f"{per} timesteps (40..{40 + per - 1}) of {wl['name']} per step, C oracle on {cores} threads"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "large-sparse", "neurons": wl["n"], "synapses": int(len(wl["pre"])),
                   "max_delay": 16, "timesteps_per_step": per, "parallelism": "replicas"},
        "timesteps_per_s": per * len(times) / sum(times),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--timesteps", type=int, default=TIMESTEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the dense, STDP and batched measurements beside the headline")
    ap.add_argument("--record-traffic", nargs=3, metavar=("CSV", "KERNEL", "WORKLOAD"),
                    help="write the DRAM traffic of KERNEL on WORKLOAD from an ncu CSV into "
                         "profiles/dram_traffic.txt and exit")
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(*args.record_traffic)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))

    from paper_2305_02510_gb300 import workloads as W

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, W.large_sparse(integer=False), rank)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as G
    if rank == 0:
        G.build()
    if world > 1:
        dist.barrier()
    from paper_2305_02510_gb300 import sn as S

    T = args.timesteps
    wl = W.large_sparse(integer=False, steps=T)
    wl["poisson"]["seed"] = replica_seed(wl["poisson"]["seed"], rank)   # own input per replica
    stream = torch.cuda.current_stream()
    ctx = S.from_workload(wl, record_steps=T, stream=stream.cuda_stream)
    n = wl["n"]
    m = int(len(wl["pre"]))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    # the public autotuner times push and pull propagation on this network's
    # own input over a whole run and keeps the faster
    S.sn_autotune(ctx, T)
    pull = S.sn_get_propagation(ctx) == S.SN_PULL

    def one(record):
        S.sn_reset(ctx)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.sn_run(ctx, T)
        b.record(stream)
        S.sn_sync(ctx)
        _, spk, ev = S.sn_get_counters(ctx)
        record.append((a.elapsed_time(b), spk, ev))

    clk = Clocks(local).start()
    for _ in range(args.warmup):
        one([])
    res = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.mark_start()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        one(res)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clk.mark_end()
    clk.stop()
    if world > 1:
        dist.barrier()
    ms = sum(r[0] for r in res) / len(res)
    spikes = sum(r[1] for r in res) / len(res)
    events = sum(r[2] for r in res) / len(res)
    # end to end through the public API with host buffers: install the input
    # (host arrays -> device), reset, run, read the raster back into pinned
    # host memory and the counters
    raster_host = torch.empty((T, ctx.words), dtype=torch.int32, pin_memory=True)
    po = wl["poisson"]
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    e_events = 0
    for _ in range(args.steps):
        S.sn_set_poisson(ctx, po["neuron"], po["rate"], po["amplitude"], po["seed"])
        S.sn_reset(ctx)
        S.sn_run(ctx, T)
        S.sn_get_spikes(ctx, 0, T, out=raster_host.numpy())
        e_events += S.sn_get_counters(ctx)[2]
    e2e_s = time.perf_counter() - e0

    ms_all, ev_all, e2e_all, e2e_ev_all = combine_ranks(ms, events, e2e_s, e_events, world,
                                                         torch.device("cuda"))
    value = ev_all / (ms_all / 1e3)

    if rank == 0:
        peak, src = peaks()
        # the method's event-proportional bytes; pull also streams every
        # synapse every step, which is reported beside it
        abytes = event_bytes(n, T, spikes, events)
        form_bytes = algorithmic_bytes_pull(n, m, T) if pull else algorithmic_bytes(n, T, spikes, events)
        kernel = "sparse_pull_kernel<SN_F32>" if pull else "sparse_reg_kernel<SN_F32>"
        achieved = abytes / (ms / 1e3) / 1e9
        traffic, traffic_src = recorded_traffic(kernel, f"large-sparse T={T}")
        store = None
        if pull:
            fmt, sbytes, sentries = S.sn_pull_store_info(ctx)
            store = {"form": "coded" if fmt == S.SN_PULL_CODED else "plain", "bytes": sbytes, "entries": sentries}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "large-sparse", "neurons": n, "synapses": m,
                       "max_delay": 16, "timesteps_per_step": T, "input": "Poisson 0.05/step into 1000 neurons",
                       "propagation": "pull" if pull else "push",
                       "l2": "256 MiB buffer written before every timed run (L2 flushed)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "timesteps_per_s": world * T / (ms_all / 1e3),
            "spikes_per_step": spikes, "events_per_step": events,
            "wall_ms_per_step": 1e3 * wall / args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": src,
                         "traffic": traffic, "traffic_source": traffic_src,
                         "kernel": kernel,
                         "algorithmic_bytes_per_launch": abytes,
                         "bytes_model": "event-proportional: 16 B per spike (row bounds), 16 B per synaptic "
                                        "event (synapse + accumulate), 56 B state and a raster bit per "
                                        "neuron and timestep",
                         "pull_store": store,
                         "kernel_bound": (f"l2+barrier: the pull store of incoming synapses "
                                          f"({store['bytes'] / 1e6:.0f} MB) stays in the L2; each timestep "
                                          f"streams it from L2 once, then one grid barrier")
                                         if pull else "l2 atomics: scattered accumulates into the pending-input "
                                                      "ring, L2-resident",
                         "form_bytes_per_launch": form_bytes,
                         "frac_form_bytes": form_bytes / (ms / 1e3) / 1e9 / peak,
                         "form_bytes_model": "pull: 8 B per synapse every timestep + 40 B state and a raster "
                                             "bit per neuron and timestep" if pull else "push: as above"},
            "e2e": {"value": e2e_ev_all / e2e_all, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": T * ctx.words * 4 + 32},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
        }
        if not args.no_extras and world == 1:
            other = S.SN_PUSH if pull else S.SN_PULL
            try:
                S.sn_set_propagation(ctx, other)
                o_ms, o_spk, o_ev = timed_runs(S, torch, stream, flush, ctx, T, 3)
                o_bytes = algorithmic_bytes(n, T, o_spk, o_ev) if pull else algorithmic_bytes_pull(n, m, T)
                alt = {"propagation": "push" if pull else "pull", "ms_per_step": o_ms,
                       "value": o_ev / (o_ms / 1e3), "unit": UNIT,
                       "kernel": "sparse_reg_kernel<SN_F32>" if pull else "sparse_pull_kernel<SN_F32>",
                       "roofline_frac": o_bytes / (o_ms / 1e3) / 1e9 / peak}
            except S.SnError as e:
                alt = {"unavailable": str(e)}
            line["extra"] = {"large_sparse_other_propagation": alt}
            line["extra"].update(extras(S, W, torch, stream, flush))
        if not args.no_cpu_baseline:
            samp = oracle_sample(wl)
            many = samp[max(samp)]
            line["cpu_baseline"] = {"value": many["value"], "unit": UNIT, "cores": many["cores"],
                                    "kind": "oracle", "sample": many["sample"],
                                    "timesteps_per_s": many["timesteps_per_s"],
                                    "host_cores": host_cores(),
                                    "single_thread": {"value": samp[1]["value"], "unit": UNIT, "cores": 1,
                                                      "timesteps_per_s": samp[1]["timesteps_per_s"]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
