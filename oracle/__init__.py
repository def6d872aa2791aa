"""CPU FP64 oracle for the gain-dissipative algorithm (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The product library never calls it.
"""
from .gda_oracle import *  # noqa: F401,F403
