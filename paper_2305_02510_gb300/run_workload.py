"""Run one named synthetic workload through the library and print its timing.

    python -m paper_2305_02510_gb300.run_workload --workload large-dense --steps 50

Workloads: large-sparse, large-dense, large-dense-stdp, batched, shared-dense,
bptt.  --scale shrinks the workload where that is meaningful (batched: number
of networks; large-dense and shared-dense: neurons) so that a profiler can
capture a launch in seconds.  Used for timing and for ncu captures; it runs
the CUDA library only.
"""

from __future__ import annotations

import argparse
import json
import time

import torch

from . import sn as S
from . import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True,
                    choices=["large-sparse", "large-dense", "large-dense-stdp", "batched", "shared-dense", "bptt"])
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--propagation", choices=["push", "pull"], default="push",
                    help="large-sparse: push or pull propagation")
    ap.add_argument("--pull-form", choices=["auto", "plain", "coded"], default="auto",
                    help="large-sparse with pull: the pull store's form (SN_PULL_PLAIN / SN_PULL_CODED)")
    ap.add_argument("--synapses-per-neuron", type=int, default=100,
                    help="large-sparse: incoming synapses per neuron (k)")
    ap.add_argument("--dense-slab", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="large-dense: column slab of 32 * k columns per block (SN_DENSE_SLAB; 0 = the library's choice)")
    args = ap.parse_args()
    import __graft_entry__ as G
    G.build()
    stream = torch.cuda.current_stream()
    T = args.steps
    wl_name = args.workload
    if wl_name == "bptt":
        from . import bptt
        task = W.bptt_task()
        net = bptt.FFNet.from_task(task)
        x = torch.tensor(task["input"], device="cuda")
        labels = torch.tensor(task["labels"], device="cuda")
        ws = [torch.tensor(w, device="cuda", requires_grad=True) for w in task["w"]]
        times = []
        for _ in range(args.repeat):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            counts = bptt.SNNFunction.apply(net, x, *ws)
            torch.nn.functional.cross_entropy(counts, labels).backward()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        print(json.dumps({"workload": wl_name, "ms": 1e3 * min(times)}))
        return
    if wl_name == "large-sparse":
        form = {"auto": 0, "plain": S.SN_PULL_PLAIN, "coded": S.SN_PULL_CODED}[args.pull_form]
        ctx = S.from_workload(W.large_sparse(k=args.synapses_per_neuron, steps=T), record_steps=T, stream=stream.cuda_stream, flags=form)
        S.sn_set_propagation(ctx, S.SN_PULL if args.propagation == "pull" else S.SN_PUSH)
    elif wl_name in ("large-dense", "large-dense-stdp"):
        n = int(16384 * args.scale) // 32 * 32
        ctx = S.from_workload(W.large_dense(n=n, stdp=wl_name.endswith("stdp"), steps=T), record_steps=T,
                              stream=stream.cuda_stream,
                              flags=S.SN_DENSE_SLAB(args.dense_slab) if args.dense_slab else S.SN_AUTO)
    elif wl_name == "batched":
        nets = W.batched_nets(count=max(1, int(4096 * args.scale)), steps=T)
        ctx = S.from_batch_workloads(nets, record_steps=T, stream=stream.cuda_stream)
    else:
        n = max(128, int(8192 * args.scale) // 128 * 128)
        ctx = S.from_shared_workload(W.shared_dense_i8(n=n, steps=T), record_steps=T, stream=stream.cuda_stream)
    times = []
    for _ in range(args.repeat):
        S.sn_reset(ctx)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.sn_run(ctx, T)
        b.record(stream)
        S.sn_sync(ctx)
        times.append(a.elapsed_time(b))
    steps, spikes, events = S.sn_get_counters(ctx)
    out = {"workload": wl_name, "steps": T, "ms": min(times), "spikes": spikes, "events": events}
    if wl_name == "large-sparse" and args.propagation == "pull":
        out["pull_store"] = dict(zip(("format", "bytes", "entries"), S.sn_pull_store_info(ctx)))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
