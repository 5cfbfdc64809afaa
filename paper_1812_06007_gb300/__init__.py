"""purl -- PowerURV (arXiv:1812.06007) on GB300.

The compute path is the C-ABI library ``libpurl.so`` (hand-written CUDA for
sm_103a, declared in ``include/purl.h``).  ``binding`` is a thin ctypes layer
with the same entry-point names; ``workloads`` synthesises seeded inputs.
Nothing here falls back to the CPU: if the library is missing, the binding
raises.
"""
__all__ = ["binding", "workloads", "autograd", "batched"]
