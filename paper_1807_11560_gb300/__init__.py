"""GB300 library for band-limited Jacobi PDE-EPDiff LDDMM with Gauss-Newton-Krylov
(Hernandez, arXiv:1807.11560).

The compute path is the C-ABI shared library ``liblddmm.so`` (CUDA for
sm_103a, built by ``paper_1807_11560_gb300.build``); ``Context`` is its thin
Python binding and ``inputs`` holds the seeded synthetic phantoms.
"""

from .lddmm import Context, LddmmError, batch_gn_solve, lib  # noqa: F401
from . import inputs  # noqa: F401
