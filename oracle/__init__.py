"""FP64 CPU oracle of the IMPM substep (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
