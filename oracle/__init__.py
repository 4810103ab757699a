"""FP64 CPU oracle (test infrastructure only; see grf_oracle.py).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and reference
legs may import this package.  The CUDA library never calls it.
"""
from .grf_oracle import *  # noqa: F401,F403
