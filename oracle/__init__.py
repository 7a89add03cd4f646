"""FP64 CPU oracle for the adaptive 2-D FMM (test infrastructure only).

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package.  It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
