"""GB300-native time-stepped spiking-network simulator (LIF neurons, delayed
synapses, external spikes, pair-based STDP).

The compute path is the C-ABI library `libsn.so` built from `csrc/` for
sm_103a; `paper_2305_02510_gb300.sn` is its thin Python binding.  Importing
this package does not load the library; the first call into `sn` does, and
raises if the library has not been built.
"""

__all__ = ["sn", "workloads", "build"]
