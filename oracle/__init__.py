"""FP64 CPU oracle of the FIRM hot path -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct statement of what the
CUDA path computes.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference legs may import it; the product path never does, and
it shares no code, tables or constants with the CUDA library.

Every function cites the passage of Wang, Shkolnisky & Singer, "A Fourier-based
Approach for Iterative 3D Reconstruction from Cryo-EM Images" (FIRM) it follows.
Where the paper is ambiguous the module docstring of `firm` states the reading
taken.  Parity of every function is pinned by tests against facts fixed
outside the oracle (closed forms, library routines, invariants, the paper's
printed numbers); `lpre` (the learned-preconditioner target and network) is
pinned by finite differences and an exact-solve special case.
"""
from .firm import *  # noqa: F401,F403
