"""FP64 CPU oracle for Iterative Least Squares (ILS) smoothing.

Test infrastructure only: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the product library never does.
It shares no code with the CUDA path.
"""
from .ils_oracle import *  # noqa: F401,F403
