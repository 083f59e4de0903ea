"""FP64 CPU oracle for the state-vector hot path of arXiv 2403.02512.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import, call or execute anything
in this package.  The CUDA path never does, and this package imports nothing
from it: the two share no code, header, helper or constant.

Modules
-------
core         gate matrices (Sec. 2.1, Eq. 1, Listing 1), generators, forward
             pass, Pauli-sum expectation values, the adjoint Jacobian and VJP,
             parameter-shift and finite-difference gradients.  State loops run
             in ``sv_oracle.c`` (plain loops over every index, FP64).
dense        independent dense Kronecker-product reference for n <= 8.
enumeration  Alg. 1 / Alg. 2 index enumerations, used only to test them.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, the printed IsingXX matrix (Eq. 1), Listing 1 semantics, brute
force and the dense reference.
"""

from .core import *  # noqa: F401,F403
