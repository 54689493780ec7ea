"""GB300 (sm_103a) Dichotomy solver for tridiagonal Toeplitz systems (arXiv 1002.2469).

The compute path is the CUDA library ``libdichotomy.so`` (C ABI in include/dichotomy.h);
this package is its Python binding.  Importing it loads (building if needed) the library
and fails loudly if that is impossible: there is no CPU fallback.
"""
from ._lib import DichotomyError, load as _load_library  # noqa: F401

_load_library()

from .dichotomy import *  # noqa: E402,F401,F403
from .dichotomy import __all__ as _dich_all  # noqa: E402

__all__ = list(_dich_all)
__version__ = "0.1.0"
