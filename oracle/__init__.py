"""CPU FP64 oracle for the POD-2G-PCG solver (arXiv 2207.02543, Algorithms 1-3, Section 3.3).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
CPU-baseline leg of bench.py, never by the solver library. It shares no code with
the CUDA path. Parity status per routine: all routines are pinned by tests in
tests/test_oracle_pins.py (closed forms, dense-matrix identities, brute-force
Krylov minimisation, textbook special cases); none is "parity unpinned".
"""
from .pod2g_oracle import *  # noqa: F401,F403
from . import pod2g_oracle  # noqa: F401
