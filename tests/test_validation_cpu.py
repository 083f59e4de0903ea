"""Host validation of the state-level C-ABI calls, without a GPU.

Every call below is given one bad argument and must return SV_ERR_ARG with a
message before it touches the device (the boundary's contract: arguments are
checked before any launch, and a rejected call leaves the state as it was).
The state is borrowed (sv_create_from_device_ptr) at an address that is never
dereferenced: every call here is rejected on the host.  The module runs only
where no GPU can be reached, so that a check that let a call through could
not send a kernel to that address.
"""

import ctypes
import math

import numpy as np
import pytest

from paper_2403_02512_gb300 import _lib as L
from workloads import Op, Term


def _gpu_reachable():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover - torch is installed wherever the tests run
        return False


pytestmark = pytest.mark.skipif(_gpu_reachable(), reason="borrows a never-dereferenced device address; "
                                                         "runs only where no GPU can be reached")

FAKE = 1 << 24  # 256-byte aligned, never dereferenced
N = 4


def _rejects(fn, *args, msg, status=1):
    with pytest.raises(L.SvError) as ei:
        fn(*args)
    assert ei.value.status == status, str(ei.value)
    assert msg in str(ei.value), str(ei.value)


@pytest.fixture
def state():
    h = L.sv_create_from_device_ptr(N, L.SV_C128, FAKE)
    yield h
    # still unlatched after every rejection: a further bad call is SV_ERR_ARG, not SV_ERR_STATE
    _rejects(L.sv_reset, h, 1 << N, msg="basis index")
    assert L.sv_info(h) == (N, L.SV_C128, FAKE)
    L.load().sv_destroy(ctypes.c_void_p(h))  # borrowed: frees nothing


def test_borrowed_state_creation_checks_its_arguments():
    _rejects(L.sv_create_from_device_ptr, N, L.SV_C128, 0, msg="NULL")
    _rejects(L.sv_create_from_device_ptr, N, L.SV_C128, FAKE + 16, msg="256-byte aligned")
    _rejects(L.sv_create_from_device_ptr, 0, L.SV_C128, FAKE, msg="outside [1, 34]")
    _rejects(L.sv_create_from_device_ptr, 35, L.SV_C64, FAKE, msg="outside [1, 34]")
    _rejects(L.sv_create_from_device_ptr, N, 2, FAKE, msg="unknown dtype")


def test_state_settings_are_checked(state):
    assert L.sv_info(state) == (N, L.SV_C128, FAKE)
    _rejects(L.sv_reset, state, 1 << N, msg="basis index")
    _rejects(L.sv_set_compute, state, 7, msg="unknown compute mode")
    assert L.load().sv_set_renormalize(ctypes.c_void_p(state), 2) == 1  # the binding passes 0 / 1 only
    assert b"0 or 1" in L.load().sv_last_error()
    _rejects(L.sv_set_workspace, state, FAKE + 8, 1024, msg="256-byte aligned")
    h64 = L.sv_create_from_device_ptr(N, L.SV_C64, FAKE)
    try:
        _rejects(L.sv_set_compute, h64, L.SV_COMPUTE_DOUBLE_FLOAT, msg="complex128 states only")
    finally:
        L.load().sv_destroy(ctypes.c_void_p(h64))


def test_single_gates_are_checked_before_any_launch(state):
    _rejects(L.sv_apply, state, L.KIND["RX"], [N], [0.1], msg="out of range")
    _rejects(L.sv_apply, state, L.KIND["RX"], [-1], [0.1], msg="out of range")
    _rejects(L.sv_apply, state, L.KIND["RX"], [0], None, msg="angles is NULL")
    _rejects(L.sv_apply, state, L.KIND["RX"], [0], [math.nan], msg="not finite")
    _rejects(L.sv_apply, state, L.KIND["Rot"], [0], [0.1, math.inf, 0.2], msg="not finite")
    _rejects(L.sv_apply, state, L.KIND["SWAP"], [1, 1], msg="used twice")
    _rejects(L.sv_apply, state, L.KIND["IsingXX"], [1], [0.3], msg="takes 2 target wires")
    _rejects(L.sv_apply, state, 99, [0], msg="unknown op kind")
    _rejects(L.sv_apply, state, L.KIND["QubitUnitary"], [0], msg="use sv_apply_matrix")
    lib = L.load()
    wires = (ctypes.c_int * 8)(*range(8))
    assert lib.sv_apply(ctypes.c_void_p(state), L.KIND["Hadamard"], wires, 7, None, 0) == 1  # > SV_MAX_TARGETS


def test_matrices_and_controls_are_checked(state):
    U = np.eye(4, dtype=np.complex128)
    U[1, 2] = complex(math.nan, 0.0)
    _rejects(L.sv_apply_matrix, state, [0, 1], U, msg="not finite")
    _rejects(L.sv_apply_matrix, state, [0, 0], np.eye(4), msg="used twice")
    _rejects(L.sv_apply_matrix, state, [0, N], np.eye(4), msg="out of range")
    lib = L.load()
    wires = (ctypes.c_int * 8)(*range(8))
    m = np.eye(128, dtype=np.complex128).view(np.float64)
    assert lib.sv_apply_matrix(ctypes.c_void_p(state), wires, 7, m.ctypes.data_as(L._dp), 0) == 1
    assert lib.sv_apply_matrix(ctypes.c_void_p(state), wires, 0, m.ctypes.data_as(L._dp), 0) == 1
    # an op whose matrix data would lie past the end of the given entries (offsets near the
    # top of the int64 range must not wrap around)
    for off in (1, 2**62, 2**63 - 2):
        op = L.SvOp()
        op.kind = L.KIND["QubitUnitary"]
        op.n_targets = 1
        op.targets[0] = 0
        op.param_index[0] = op.param_index[1] = op.param_index[2] = -1
        op.scale = 1.0
        op.matrix_offset = off
        data = np.eye(2, dtype=np.complex128).view(np.float64)
        tape = L.SvTape(1, ctypes.pointer(op), 0, data.ctypes.data_as(L._dp), 4)
        assert lib.sv_forward(ctypes.c_void_p(state), ctypes.byref(tape), None) == 1
        assert b"out of range" in lib.sv_last_error()
    # controls: a repeated wire, a control value other than 0 / 1, too many controls
    for bad, msg in ((Op("PauliX", (0,), controls=(0,)), "used twice"),
                     (Op("PauliX", (0,), controls=(1,), control_values=(2,)), "control value"),
                     (Op("RY", (0,), (0,), controls=(N,)), "out of range")):
        _rejects(L.sv_forward, state, L.Tape([bad], 1), np.zeros(1), msg=msg)
    op = L.Tape([Op("PauliX", (0,))], 0)
    op.ops[0].n_controls = 9
    _rejects(L.sv_forward, state, op, np.zeros(0), msg="n_controls")


def test_observables_are_checked(state):
    def sums(*obs):
        return L.PauliSums(list(obs))

    _rejects(L.sv_expval, state, sums([Term(1.0, ((N, "Z"),))]), msg="acts on a wire >= n")
    _rejects(L.sv_expval, state, sums([Term(math.nan, ((0, "Z"),))]), msg="coefficient not finite")
    _rejects(L.sv_var, state, sums([Term(1.0, ((0, "X"),))], [Term(1.0, ((N + 3, "Y"),))]),
             msg="observable 1 term 0 acts on a wire >= n")
    lib = L.load()
    bad = L.SvPauliSum(-1, None, None, None)
    out = np.zeros(1)
    assert lib.sv_expval(ctypes.c_void_p(state), ctypes.byref(bad), 1, L._dptr(out)) == 1
    assert b"n_terms < 0" in lib.sv_last_error()
    nulls = L.SvPauliSum(2, None, None, None)
    assert lib.sv_expval(ctypes.c_void_p(state), ctypes.byref(nulls), 1, L._dptr(out)) == 1
    assert b"NULL term arrays" in lib.sv_last_error()
    ok = sums([Term(1.0, ((0, "Z"),))])
    assert lib.sv_expval(ctypes.c_void_p(state), ok.array, 1, None) == 1  # out is NULL


def test_measurements_are_checked(state):
    _rejects(L.sv_probs, state, [N], msg="outside")
    _rejects(L.sv_probs, state, [1, 1], msg="repeated")
    _rejects(L.sv_probs, state, list(range(N + 1)), msg="wires outside")
    _rejects(L.sv_sample, state, [0], [0.5, 1.0], msg="not in [0, 1)")
    _rejects(L.sv_sample, state, [0], [math.nan], msg="not in [0, 1)")
    _rejects(L.sv_sample, state, [0], [-0.25], msg="not in [0, 1)")


def test_circuits_and_gradients_are_checked(state):
    tape = L.Tape([Op("RX", (0,), (0,)), Op("RY", (1,), (1,))], 2)
    obs = L.PauliSums([[Term(1.0, ((0, "Z"),))]])
    _rejects(L.sv_forward, state, tape, np.array([0.1, math.nan]), msg="parameter 1 is not finite")
    _rejects(L.sv_forward, state, L.Tape([Op("RX", (0,), (2,))], 2), np.zeros(2), msg="param_index 2 >= n_params 2")
    _rejects(L.sv_adjoint_jacobian, state, tape, np.array([math.inf, 0.0]), obs, msg="parameter 0 is not finite")
    _rejects(L.sv_adjoint_jacobian, state, tape, np.zeros(2), L.PauliSums([]), msg="at least one observable")
    _rejects(L.sv_adjoint_vjp, state, tape, np.zeros(2), obs, [math.nan], msg="grad_out[0] is not finite")
    lib = L.load()
    neg = L.SvPauliSum(-3, None, None, None)
    g = np.ones(1)
    out = np.zeros(2)
    p = np.zeros(2)
    assert lib.sv_adjoint_vjp(ctypes.c_void_p(state), ctypes.byref(tape.struct), L._dptr(p), ctypes.byref(neg), 1,
                              L._dptr(g), L._dptr(out)) == 1
    assert b"n_terms < 0" in lib.sv_last_error()
    neg_tape = L.SvTape(-1, None, 0, None, 0)
    assert lib.sv_forward(ctypes.c_void_p(state), ctypes.byref(neg_tape), None) == 1
    assert b"negative tape sizes" in lib.sv_last_error()
    ph = ctypes.c_void_p()
    bad = L.Tape([Op("PauliX", (0,), controls=(1,), control_values=(3,))], 0)
    assert lib.sv_program_create(ctypes.c_void_p(state), ctypes.byref(bad.struct), None, 0, ctypes.byref(ph)) == 1
    assert ph.value is None


def test_sparse_observables_are_checked_on_the_host():
    rows = 1 << N
    ip = np.arange(rows + 1, dtype=np.int64)
    ix = np.arange(rows, dtype=np.int64)
    v = np.ones(rows, dtype=np.complex128)
    for bad_ip, bad_ix, bad_v, msg in (
            (ip + 1, ix, v, "indptr must run from 0 to nnz"),
            (np.concatenate([[0, 2, 1], ip[3:]]), ix, v, "indptr decreases"),
            (ip, np.where(ix == 5, rows, ix), v, "column index"),
            (ip, ix, np.where(ix == 3, complex(math.inf, 0), v), "not finite")):
        with pytest.raises(L.SvError) as ei:
            L.Sparse(N, bad_ip, bad_ix, bad_v)
        assert ei.value.status == 1 and msg in str(ei.value)


def test_batches_are_checked_on_the_host():
    from workloads import Circuit

    def circ(n, ops, n_params=0, obs=None, basis=0):
        return Circuit(n, ops, n_params, [obs if obs is not None else [Term(1.0, ((0, "Z"),))]], basis)

    good = circ(3, [Op("Hadamard", (0,))])
    for bad, status, msg in (
            (circ(31, [Op("Hadamard", (0,))]), 1, "outside [1, 30]"),
            (circ(3, [Op("RX", (3,), (0,))], 1), 1, "batch circuit 1 op 0: target wire 3 out of range"),
            (circ(3, [Op("Hadamard", (0,))], obs=[Term(1.0, ((1, "X"),))]), 5, "Z-only"),
            (circ(3, [Op("Hadamard", (0,))], obs=[Term(1.0, ((3, "Z"),))]), 1, "bad Z word"),
            (circ(3, [Op("Hadamard", (0,))], obs=[Term(math.nan, ((0, "Z"),))]), 1, "bad Z word"),
            (circ(3, [Op("Hadamard", (0,))], basis=8), 1, "basis state out of range")):
        with pytest.raises(L.SvError) as ei:
            L.Batch([good, bad], L.SV_C64)
        assert ei.value.status == status and msg in str(ei.value), str(ei.value)
    with pytest.raises(L.SvError) as ei:
        L.Batch([good], 3)
    assert ei.value.status == 1 and "unknown dtype" in str(ei.value)
