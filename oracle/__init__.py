"""FP64 CPU oracle of the two-timescale multicomponent lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only the tests, the smoke check and the CPU-baseline leg of the benchmark may
call it.  It shares no code, table or constant with the CUDA library.

Every function follows the paper (Monteferrante, Melchionna, Marini Bettolo
Marconi, "Lattice Boltzmann Method for mixtures at variable Schmidt number")
step by step, in the paper's order and notation, and says which passage it
restates.  All pins (closed forms, invariants, brute force) live in
``tests/test_oracle_*.py``.  No function here is "parity unpinned".
"""

from .lbm_oracle import *  # noqa: F401,F403
