"""GB300-native state-vector core: gates, Pauli-sum expectation values and the
adjoint-method Jacobian of arXiv 2403.02512, as hand-written CUDA for sm_103a
behind the C ABI in include/sv.h.

``_lib`` binds that ABI with the same function names; ``torch_api`` adds
torch-memory state vectors, planned programs and an autograd function.
"""

from . import _lib  # noqa: F401
from ._lib import (SV_C64, SV_C128, KIND, PauliSums, SvError, Tape, load,  # noqa: F401
                   sv_adjoint_jacobian, sv_adjoint_vjp, sv_apply, sv_apply_matrix, sv_apply_op,
                   sv_create, sv_create_from_device_ptr, sv_destroy, sv_expval, sv_forward,
                   sv_get_state, sv_info, sv_norm2, sv_plan_query, sv_program_create,
                   sv_program_destroy, sv_program_expval, sv_program_forward, sv_program_jacobian,
                   sv_program_set_params, sv_program_stats, sv_program_vjp, sv_reset,
                   sv_set_alloc_cap, sv_set_state, sv_set_stream, sv_set_workspace,
                   sv_synchronize, sv_version)


def __getattr__(name):
    # torch-facing classes load lazily so the ctypes layer imports without torch
    if name in ("StateVector", "Program", "AdjointExpval", "expval"):
        from . import torch_api
        return getattr(torch_api, name)
    raise AttributeError(name)
