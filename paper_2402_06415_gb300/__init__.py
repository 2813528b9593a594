"""GB300-native checkerboard Metropolis sweep of the 2D Ising model.

The hot path of arXiv 2402.06415 (the bipartite Monte Carlo sweep of Results A
and the Supplementary MC details), restated for the square-lattice Ising
model, runs in hand-written CUDA kernels for sm_103a behind the C-ABI of
``include/ising.h`` (``libising.so``).  This package is the thin Python
binding (same entry-point names) plus host-side statistics.  Nothing here falls
back to the CPU: without the CUDA library every call raises.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import EXPORTED, IsingError, Lattice, lib  # noqa: F401
