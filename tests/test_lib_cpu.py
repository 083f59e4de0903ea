"""Host-only checks of libsv.so: it builds for sm_103a, loads, exports every
entry point declared in include/sv.h, and its planner / validation work
without a GPU."""

import os
import re

import numpy as np
import pytest

import paper_2403_02512_gb300 as svlib
from paper_2403_02512_gb300 import _lib as L
from workloads import (Op, layered_circuit, qaoa_maxcut, random_circuit, ry_cz_brick, strongly_entangling,
                       vqe_givens)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "sv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = L.load()
    syms = _declared_symbols()
    assert len(syms) >= 25
    for name in syms:
        assert hasattr(lib, name), f"libsv.so does not export {name}"
        assert name in L.PROTOTYPES, f"binding has no prototype for {name}"
    assert "sm_103a" in svlib.sv_version()


def test_plan_counts_fuse_gates_into_few_passes():
    c, _ = strongly_entangling(24, 8)
    tape = L.Tape(c.ops, c.n_params)
    f128, a128 = L.sv_plan_query(24, L.SV_C128, tape)
    f64, a64 = L.sv_plan_query(24, L.SV_C64, tape)
    n_gates = len(c.ops)
    assert f128 < n_gates / 4 and f64 <= f128
    assert a128 < 3 * n_gates / 4  # expanded Rot = 3 ops each
    c1, _ = layered_circuit(12, 10)
    f, a = L.sv_plan_query(12, L.SV_C128, L.Tape(c1.ops, c1.n_params))
    assert f <= 2 * 10 and a >= 1  # 12 wires > 11 local bits: two passes per layer


@pytest.mark.parametrize("maker", ["qaoa", "vqe", "rycz"])
def test_plan_query_accepts_every_workload_shape(maker):
    if maker == "qaoa":
        c = qaoa_maxcut(20, 4)
    elif maker == "vqe":
        c, _ = vqe_givens(24, 12, 40, 120, 10)
    else:
        c, _ = ry_cz_brick(30, 20)
    f, a = L.sv_plan_query(c.n, L.SV_C128, L.Tape(c.ops, c.n_params))
    assert 1 <= f <= len(c.ops) and 1 <= a


@pytest.mark.parametrize("bad,msg", [
    (Op("RX", (5,), (0,)), "out of range"),
    (Op("PauliX", (1,), controls=(1,)), "used twice"),
    (Op("RX", (0,), (3,)), "n_params"),
])
def test_validation_rejects_bad_ops_before_any_launch(bad, msg):
    tape = L.Tape([bad], 1)
    with pytest.raises(L.SvError) as ei:
        L.sv_plan_query(4, L.SV_C128, tape)
    assert ei.value.status == 1 and msg in str(ei.value)


def test_validation_rejects_bad_sizes():
    tape = L.Tape([Op("Hadamard", (0,))], 0)
    for n in (0, 35):
        with pytest.raises(L.SvError) as ei:
            L.sv_plan_query(n, L.SV_C128, tape)
        assert ei.value.status == 1


def test_planner_checks_hold_for_random_circuits():
    # check_plan runs inside sv_plan_query: local targets, tile widths, low runs
    for n in list(range(1, 16)) + [20, 24, 30]:
        for seed in range(4):
            c, _ = random_circuit(n, 60, 1000 * n + seed, max_controls=3)
            for dt in (L.SV_C64, L.SV_C128):
                f, a = L.sv_plan_query(n, dt, L.Tape(c.ops, c.n_params))
                assert 1 <= f <= len(c.ops) and a >= f


# ---- planner features, described without a GPU ------------------------------
def test_plan_describe_qaoa_cost_layers_become_phase_runs_and_mixers_multi_ops():
    from workloads import qaoa_maxcut
    c = qaoa_maxcut(20, 4)
    fwd, adj = L.sv_plan_describe(20, L.SV_C64, L.Tape(c.ops, c.n_params))
    assert fwd["phase_run"] == 4                      # one diagonal per cost layer (30 RZZ each)
    assert fwd["diag"] == 0                           # no RZZ left as its own micro-op
    assert fwd["multi"] >= 4 * 20 // 3                # mixers: up to 3 RX per barrier
    # the adjoint keeps each cost layer as one trainable phase run (one Jacobian slot per layer);
    # the adjoint keeps each cost layer as one trainable phase run (one Jacobian slot per layer)
    assert adj["phase_run"] == 4 and adj["diag"] == 0 and adj["multi"] == 0


def test_plan_describe_rot_runs_fuse_in_both_plans():
    c, _ = strongly_entangling(12, 2, seed=3)
    fwd, adj = L.sv_plan_describe(12, L.SV_C128, L.Tape(c.ops, c.n_params))
    # the adjoint expands Rot into RZ, RY, RZ and fuses them back: one block per Rot
    assert adj["fused_run"] == 2 * 12
    assert fwd["dense"] == 0 and adj["dense"] == 0


def test_plan_describe_counts_are_consistent_with_pass_counts():
    for seed in range(5):
        c, _ = random_circuit(10, 60, seed, max_controls=2)
        tape = L.Tape(c.ops, c.n_params)
        fwd, adj = L.sv_plan_describe(10, L.SV_C128, tape)
        f, a = L.sv_plan_query(10, L.SV_C128, tape)
        assert fwd["passes"] + fwd["wide_dense"] == f and adj["passes"] + adj["wide_dense"] == a


def test_plan_describe_dense_blocks_of_the_30_qubit_workload_are_wide_steps():
    # four 5-qubit dense blocks: steps outside the tiles in both plans; the
    # 290 CZ gates of the brick are diagonal micro-ops; all 600 RY are trained
    c, _ = ry_cz_brick(30, 20)
    for dt in (L.SV_C64, L.SV_C128):
        fwd, adj = L.sv_plan_describe(30, dt, L.Tape(c.ops, c.n_params))
        assert fwd["wide_dense"] == 4 and adj["wide_dense"] == 4
        assert fwd["diag"] == 290 and adj["diag"] == 290
        assert fwd["dense"] == 0 and adj["dense"] == 0
        assert adj["multi"] == 0


# ---------------------------------------------------------------------------
# Hermitian observables as Pauli words (host only)
# ---------------------------------------------------------------------------
def _terms_matrix(n, terms):
    # sum_t c_t (x)_w P_w over all n wires, wire 0 leftmost (independent of the library)
    pauli = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
             "Z": np.diag([1.0, -1.0])}
    out = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t in terms:
        letters = dict(t.paulis)
        m = np.ones((1, 1))
        for w in range(n):
            m = np.kron(m, pauli[letters.get(w, "I")])
        out += t.coeff * m
    return out


@pytest.mark.parametrize("n,wires,seed", [(3, (0,), 1), (4, (2, 0), 2), (5, (1, 4, 3), 3), (6, (5, 0, 2, 3), 4),
                                          (5, (4, 2, 0, 3, 1), 5)])
def test_hermitian_to_pauli_reconstructs_the_matrix(n, wires, seed):
    from oracle import dense
    rng = np.random.default_rng(seed)
    k = len(wires)
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    A = (a + a.conj().T) / 2
    terms = L.sv_hermitian_to_pauli(n, wires, A)
    assert 1 <= len(terms) <= 4 ** k
    np.testing.assert_allclose(_terms_matrix(n, terms), dense.embed(n, list(wires), A), atol=1e-13)


def test_hermitian_to_pauli_known_matrices():
    proj1 = np.diag([0.0, 1.0])                                   # |1><1| = (I - Z) / 2
    t = sorted(L.sv_hermitian_to_pauli(4, [2], proj1), key=lambda t: len(t.paulis))
    assert [(x.coeff, x.paulis) for x in t] == [(0.5, ()), (-0.5, ((2, "Z"),))]
    zx = np.kron(np.diag([1.0, -1.0]), np.array([[0, 1], [1, 0]]))  # Z on wire 3, X on wire 1
    t = L.sv_hermitian_to_pauli(4, [3, 1], zx)
    assert [(x.coeff, x.paulis) for x in t] == [(1.0, ((1, "X"), (3, "Z")))]
    y = np.array([[0, -1j], [1j, 0]])
    t = L.sv_hermitian_to_pauli(2, [0], y)
    assert [(x.coeff, x.paulis) for x in t] == [(1.0, ((0, "Y"),))]


def test_hermitian_to_pauli_rejects_bad_input():
    with pytest.raises(L.SvError) as ei:
        L.sv_hermitian_to_pauli(3, [0], np.array([[0, 1], [0, 0]]))   # not Hermitian
    assert ei.value.status == 1 and "Hermitian" in str(ei.value)
    for wires in ([0, 0], [3], [-1]):
        with pytest.raises(L.SvError):
            L.sv_hermitian_to_pauli(3, wires, np.eye(1 << len(wires)))
    with pytest.raises(L.SvError):
        L.sv_hermitian_to_pauli(8, list(range(6)), np.eye(64))       # more than 5 wires
    with pytest.raises(L.SvError):
        L.sv_hermitian_to_pauli(3, [0], np.eye(2), tol=-1.0)


def test_hermitian_to_pauli_drops_words_at_or_below_tol():
    A = np.diag([1.0, 1.0 + 1e-9])   # I (1 + 5e-10) - 5e-10 Z
    assert len(L.sv_hermitian_to_pauli(2, [1], A)) == 2
    t = L.sv_hermitian_to_pauli(2, [1], A, tol=1e-8)
    assert len(t) == 1 and t[0].paulis == ()


def test_static_expval_rejects_bad_arguments_before_touching_a_device():
    # argument checks come before any CUDA call, so they hold without a GPU
    from workloads import Term
    ps = L.PauliSums([[Term(1.0, ((0, "Z"),))]])
    host = np.zeros(16, dtype=np.complex128)
    for ptr, n, dt, msg in ((0, 4, L.SV_C128, "NULL"), (host.ctypes.data + 8, 4, L.SV_C128, "aligned"),
                            (host.ctypes.data, 0, L.SV_C128, "n out of range"),
                            (host.ctypes.data, 4, 7, "dtype")):
        with pytest.raises(L.SvError) as ei:
            L.sv_expval_static(ptr, n, dt, ps)
        assert ei.value.status == 1 and msg in str(ei.value)
    # a host pointer never reaches a kernel: without a GPU the call ends in an error status
    with pytest.raises(L.SvError) as ei:
        L.sv_expval_static(host.ctypes.data, 4, L.SV_C128, ps)
    assert ei.value.status in (1, 3)
