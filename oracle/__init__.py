"""FP64 CPU oracle of CAC-MFZ-CDP.  Test infrastructure only: imported by
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs, never by the
product path."""
from .cac_mfz import *  # noqa: F401,F403
