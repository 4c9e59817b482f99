"""FP64 CPU oracle of the multipole shear-3PCF estimator (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import this package. The CUDA library never calls it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
