"""GB300-native (sm_103a) hot path of the sub-grid DG shallow-water method of
arXiv 2505.18743: matrix-free DG operator with pixel-resolved wet depth and
area, Rusanov fluxes with hydrostatic reconstruction, conservative tracer,
wet-dry degree switch and the IMEX Runge-Kutta stage update.

``swdg`` is the ctypes binding of the C-ABI (``include/swdg.h``) implemented
by the in-tree ``libswdg.so``; ``workloads`` generates seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "swdg"]
