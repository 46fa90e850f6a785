"""ORACLE -- test infrastructure only.

Plain FP64 CPU reference of the C-PCM/ISWIG hot path (surface, A, Bz, ESP,
Fock, LU and PCG solves, energy).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA library (``paper_1505_07851_gb300``), and neither imports the
other.
"""
from .pcm import *  # noqa: F401,F403
from .pcm import (ExpandedBasis, Preconditioner, a_matrix, boys, bz, dynamic_delta, energy, esp,
                  f_factor, fibonacci_directions, fock, fock_blocks, gradient, gradient_a,
                  gradient_bz, gradient_c, octree_blocks, pcg, prim_integrals, prim_norm,
                  rbj_blocks, run, solve_lu, splitmix64, surface, switching_factor)
