"""B300-native parallel Bayesian cross-validation (PCV, arXiv 2310.07002).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/pcv.h``); ``pcv`` is its Python binding, ``workloads`` the seeded
synthetic inputs.
"""
from . import workloads  # noqa: F401


def build_library(force: bool = False) -> str:
    """Compile the CUDA library in-tree (see the ``build`` module)."""
    from .build import build as _b
    return _b(force=force)


def PCV(*args, **kw):  # noqa: N802
    from .pcv import PCV as _P
    return _P(*args, **kw)
