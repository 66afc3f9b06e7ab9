"""GB300-native hybrid purification-METTS sampler (arXiv:1910.09142).

The sample path (init, evolve, measure, collapse) lives in the CUDA library
``_lib/libhmetts.so`` behind the C ABI of ``include/hmetts.h``.  Modules:

* ``binding``     ctypes wrapper of the C ABI (``Context``, ``params``);
* ``build``       compiles the library for sm_103a;
* ``serve``       continuous-batching server, timed request streams,
                  checkpoint and restore;
* ``estimators``  binned thermal averages of many chains, merged across ranks.
"""
from . import binding, build  # noqa: F401
