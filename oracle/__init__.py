"""CPU oracle for the TensorACO iteration -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  The GPU library never loads it and shares no code with
it.  See oracle/oracle.h for the readings of the paper it fixes.
"""
from .binding import *  # noqa: F401,F403
