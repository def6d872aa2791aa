"""GB300-native gain-dissipative solver for the XY and Ising Hamiltonians.

The compute path is the CUDA library libgda.so (C ABI in include/gda.h);
this package holds its sources (csrc/), the in-tree build (_build.py) and a
ctypes binding (gda.py).
"""
from . import gda  # noqa: F401
from .gda import (BF16, EULER, FP32, ISING, RK4, XY, GdaError, Params, Solver,  # noqa: F401
                  default_params, load_library)
