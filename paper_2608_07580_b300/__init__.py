"""B300 (sm_103a) per-pixel wildfire-temperature retrieval.

The product is the C-ABI library libfirert.so (include/firert.h) built from
csrc/ by build.py; firert.py is its ctypes binding.
"""
from . import build as _build  # noqa: F401


def load():
    """Import the binding (raises if the CUDA library is missing)."""
    from . import firert
    return firert
