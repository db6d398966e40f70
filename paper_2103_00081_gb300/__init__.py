"""GB300-native hydrothermal finite element step (matrix-free CUDA, sm_103a).

The compute path lives in the CUDA library ``libht.so`` (C ABI in
``include/ht.h``); this package holds its build script and a thin ctypes
binding.  Importing ``Simulator`` loads the library and fails loudly if it has
not been built.
"""
from ._lib import (HT_BC_DIRICHLET, HT_BC_FLUX, HT_BC_NONE, HT_FP64, HT_HEAD,  # noqa: F401
                   HT_MIXED, HT_PREC_CHEBYSHEV, HT_PREC_JACOBI, HT_QX, HT_QY, HT_QZ, HT_TEMP)


def __getattr__(name):
    if name in ("Simulator", "HTError"):
        from . import hydro
        return getattr(hydro, name)
    raise AttributeError(name)
