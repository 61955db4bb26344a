"""GB300-native short-range coarse-grained MD (ESPResSo++ hot path).

`espp` is the ctypes binding of libespp_gb.so (C ABI in include/espp.h);
`inputs` generates seeded synthetic systems.  Importing the package does not
load the CUDA library; the first call that needs it does, and raises if it is
missing.
"""
from . import espp, inputs  # noqa: F401
from .espp import System, EsppError  # noqa: F401
