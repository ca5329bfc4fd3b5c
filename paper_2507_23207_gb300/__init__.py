"""GB300 (sm_103a) Khatri-Rao random projection library: Python binding of libkrp.

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/krp.h``); this package only marshals arguments (see ``krp.py``).
"""

from .krp import *  # noqa: F401,F403
from .krp import Context, KrpError, load_library, EXPORTED, LIB_PATH  # noqa: F401

__all__ = ["Context", "KrpError", "load_library", "EXPORTED", "LIB_PATH"]
