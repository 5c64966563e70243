"""CPU float64 oracle for tensor-train contraction -- test infrastructure only.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The CUDA library never calls it.
"""
from .tt_oracle import *  # noqa: F401,F403
from .tt_oracle import __all__  # noqa: F401
