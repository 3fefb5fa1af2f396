"""Failure paths of every create call, by host-side fault injection.

With SN_FAULT_ALLOC_AT = k in the environment, the k-th device allocation of
a create call fails (nothing is allocated for it).  For k = 1, 2, ... every
create call must then return SN_ENOMEM with a message, free what it had
allocated, leave the CUDA context usable, and succeed once k exceeds its
allocation count.  No GPU fault is made: the failure is made on the host."""

import os

import numpy as np
import pytest

from paper_2305_02510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def _creators():
    from paper_2305_02510_gb300 import sn as S
    sparse = W.random_small(40, n=300, integer=False, steps=20, max_delay=4, p=0.05)
    dense = W.large_dense(n=256, steps=20)
    shared = W.shared_dense_i8(n=256, batch=128, steps=20)
    nets = W.batched_nets(count=6, steps=20, nmax=256)
    task = W.bptt_task(batch=8, sizes=(40, 48, 6), steps=20, seed=4)
    return {
        "sparse": lambda: S.from_workload(sparse, flags=S.SN_PROP_PULL),
        "axonal": lambda: S.sn_create(sparse["threshold"], sparse["leak"], sparse["reset"], sparse["refractory"],
                                      sparse["pre"], sparse["post"], sparse["weight"], sparse["delay"],
                                      max_delay=6, axonal_delay=np.ones(sparse["n"], np.int32)),
        "dense": lambda: S.from_workload(dense),
        "shared": lambda: S.from_shared_workload(shared),
        "batched": lambda: S.from_batch_workloads(nets),
        "shard": lambda: S.from_workload_shard(sparse, 32, 268),
        "ff": lambda: S.sn_create_ff(task["sizes"], task["delay"], threshold=1.0, leak=0.05, reset=0.0,
                                     refractory=0, slope=10.0, checkpoint_every=10, batch=8, steps=20),
    }


@pytest.mark.parametrize("kind", ["sparse", "axonal", "dense", "shared", "batched", "shard", "ff"])
def test_injected_allocation_failures(kind):
    from paper_2305_02510_gb300 import sn as S
    make = _creators()[kind]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for k in range(1, 200):
            os.environ["SN_FAULT_ALLOC_AT"] = str(k)
            try:
                ctx = make()
            except S.SnError as e:
                assert e.status == S.SN_ENOMEM, (k, e.status, str(e))
                assert "SN_FAULT_ALLOC_AT" in str(e)
                failures += 1
                continue
            # past the allocation count (or, for the feedforward context, a
            # failure its tensor-core setup absorbs by keeping the CUDA-core
            # engine): the context works
            del ctx
            if kind != "ff" or k > 60:
                break
    finally:
        os.environ.pop("SN_FAULT_ALLOC_AT", None)
    assert failures >= 3
    # no allocation of the failed calls is left behind, and the context still runs
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
    ctx = make()
    if kind in ("sparse", "dense", "axonal", "batched"):
        S.sn_run(ctx, 5)
        S.sn_sync(ctx)
