"""GB300-native hybrid purification-METTS sampler (arXiv:1910.09142).

The sample path (init, evolve, measure, collapse) lives in the CUDA library
``_lib/libhmetts.so`` behind the C ABI of ``include/hmetts.h``; ``binding``
is its ctypes wrapper and ``build`` compiles it for sm_103a.
"""
from . import binding, build  # noqa: F401
