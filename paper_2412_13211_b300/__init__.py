"""B300-native batched rigid-body step (C ABI in include/msh.h, kernels in csrc/)."""
from . import scenes  # noqa: F401
from .build import build as build_library  # noqa: F401


def MshSim(*args, **kwargs):
    """Constructs a `sim.MshSim` (imports torch lazily)."""
    from .sim import MshSim as _M
    return _M(*args, **kwargs)
