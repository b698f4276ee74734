"""FP64 CPU oracle for the quasi-Newton method (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline and
reference legs may import this package. The CUDA library never calls it and
shares no code with it.
"""
from .qn_oracle import *  # noqa: F401,F403
