"""CPU oracle (test infrastructure only): plain fp64 direct sums and dense solves.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs may import
this package.  It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
from . import oracle as _o

__all__ = [n for n in dir(_o) if not n.startswith("_")]
