"""GB300-native (sm_103a) finite-difference topology optimizer for permanent magnets.

After Abert et al., "A fast finite-difference algorithm for topology
optimization of permanent magnets" (arXiv:1707.09898). The compute path is the
CUDA library ``libtopomag.so`` (C ABI in ``include/topomag.h``); the Python
modules only marshal device pointers and streams.

    from paper_1707_09898_gb300 import Magnet, StrayField, TopoObjective
"""

from . import workloads  # noqa: F401  (inputs only; no method arithmetic)


def __getattr__(name):
    if name in ("Magnet", "StrayField", "TopoObjective"):
        from . import magnet
        return getattr(magnet, name)
    raise AttributeError(name)
