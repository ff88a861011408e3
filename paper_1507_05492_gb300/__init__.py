"""GB300-native scoring of community partitions (arXiv 1507.05492 metrics).

``qm`` is the binding of the CUDA library libqm.so (C ABI in include/qm.h),
``gen`` makes seeded LFR-style workloads, ``server`` is the continuous-batching
request loop.  Importing the package does not load the CUDA library; the first
call does, and fails loudly if it has not been built.
"""
from . import gen  # noqa: F401
