"""GB300-native replica-tensor-train (RTT) Monte Carlo sampler.

The compute path is librtt.so (hand-written CUDA for sm_103a, C ABI in
include/rtt.h); ``rtt`` is its thin Python binding and ``inputs`` the seeded
synthetic workload generator.  Submodules are imported lazily so that the
input generator can be used without CUDA.
"""
__all__ = ["rtt", "inputs", "build"]
