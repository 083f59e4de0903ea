"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Sources of truth: the printed IsingXX matrix (Eq. 1), Listing 1 semantics,
Alg. 1 / Alg. 2 brute force, closed forms (RX expectation values, GHZ,
product states, Hartree-Fock energies, QAOA p=1), matrix exponentials of the
generators (scipy), and the independent dense Kronecker reference.
"""

import cmath
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import dense, enumeration
from workloads import (Circuit, MatrixOp, Op, Term, GATE_ARITY, GATE_NPARAMS, layered_circuit,
                       dense_block_wires, random_unitary, qaoa_maxcut, random_circuit, random_hamiltonian, random_state,
                       regular_graph, strongly_entangling, vqe_givens, ry_cz_brick)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ONE_ANGLE = [g for g, k in GATE_NPARAMS.items() if k == 1]


# ---------------------------------------------------------------------------
# Alg. 1 / Alg. 2 enumerations (brute force)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", range(1, 11))
def test_alg1_pairs_partition_the_state(n):
    for q in range(n):
        pairs = list(enumeration.single_qubit_pairs(n, q))
        assert len(pairs) == 1 << (n - 1)
        bit = 1 << (n - 1 - q)
        flat = [i for p in pairs for i in p]
        assert sorted(flat) == list(range(1 << n))
        assert all((i0 & bit) == 0 and i1 == i0 | bit for i0, i1 in pairs)


def test_alg1_low_mask_reading_at_offset_zero():
    # q = n-1 gives q_offset = 0: the low mask must be empty (reading of the
    # printed shift by the full bit width).
    assert enumeration.gap_masks([0])[0] == 0
    pairs = list(enumeration.single_qubit_pairs(3, 2))
    assert pairs == [(0, 1), (2, 3), (4, 5), (6, 7)]


@pytest.mark.parametrize("n", range(2, 7))
def test_alg2_pairs_are_exactly_the_control_matching_pairs(n):
    rng = np.random.default_rng(n)
    for target in range(n):
        others = [w for w in range(n) if w != target]
        for nc in range(0, min(3, n - 1) + 1):
            for controls in itertools.combinations(others, nc):
                vals = [int(v) for v in rng.integers(0, 2, size=nc)]
                got = list(enumeration.controlled_pairs(n, target, controls, vals))
                alt = list(enumeration.controlled_pairs_by_insertion(n, target, controls, vals))
                assert got == alt
                tb = 1 << (n - 1 - target)
                want = []
                for i in range(1 << n):
                    if i & tb:
                        continue
                    if all(((i >> (n - 1 - c)) & 1) == v for c, v in zip(controls, vals)):
                        want.append((i, i | tb))
                assert sorted(got) == want
                assert len(got) == 1 << (n - 1 - nc)   # cost ~ 2^-c of the uncontrolled gate


@pytest.mark.parametrize("n", [3, 4, 5])
def test_alg2_enumeration_applies_the_dense_controlled_gate(n):
    rng = np.random.default_rng(100 + n)
    U = scipy.linalg.expm(1j * (lambda a: a + a.conj().T)(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))))
    for target in range(n):
        controls = [w for w in range(n) if w != target][:2]
        vals = [1, 0][:len(controls)]
        psi = random_state(n, 7 + target)
        out = psi.copy()
        for i0, i1 in enumeration.controlled_pairs(n, target, controls, vals):
            a0, a1 = psi[i0], psi[i1]
            out[i0] = U[0, 0] * a0 + U[0, 1] * a1
            out[i1] = U[1, 0] * a0 + U[1, 1] * a1
        want = dense.controlled(n, [target], U, controls, vals) @ psi
        np.testing.assert_allclose(out, want, atol=1e-14)


# ---------------------------------------------------------------------------
# Gate matrices
# ---------------------------------------------------------------------------
def _golden_isingxx(phi):
    tok = {"c": math.cos(phi / 2), "0": 0.0, "-is": -1j * math.sin(phi / 2)}
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "isingxx_eq1.txt"))
            if ln.strip() and not ln.startswith("#")]
    return np.array([[tok[t] for t in r] for r in rows], dtype=np.complex128)


@pytest.mark.parametrize("phi", [0.0, 0.3, -1.1, math.pi, 2.5, 5.9])
def test_isingxx_matches_printed_eq1(phi):
    np.testing.assert_allclose(oracle.gate_matrix("IsingXX", [phi]), _golden_isingxx(phi), atol=1e-15)


@pytest.mark.parametrize("name", list(GATE_ARITY))
def test_every_gate_is_unitary(name):
    rng = np.random.default_rng(3)
    for _ in range(5):
        M = oracle.gate_matrix(name, rng.uniform(-7, 7, size=GATE_NPARAMS[name]))
        np.testing.assert_allclose(M.conj().T @ M, np.eye(M.shape[0]), atol=1e-14)


@pytest.mark.parametrize("name", ONE_ANGLE)
def test_gate_equals_exponential_of_its_generator(name):
    G, s = oracle.generator(name)
    np.testing.assert_allclose(G, G.conj().T, atol=0)          # Hermitian generator
    for theta in (0.0, 0.4, -2.2, 3.7):
        np.testing.assert_allclose(oracle.gate_matrix(name, [theta]),
                                   scipy.linalg.expm(1j * s * theta * G), atol=1e-13)


def test_rotations_are_exp_minus_i_theta_p_over_2():
    # Reading of the RX sign: exp(-i theta/2 P) everywhere (Eq. 1 form).
    for name, P in (("RX", oracle.PX), ("RY", oracle.PY), ("RZ", oracle.PZ)):
        for t in (0.1, 1.3, -2.0):
            np.testing.assert_allclose(oracle.gate_matrix(name, [t]),
                                       scipy.linalg.expm(-0.5j * t * P), atol=1e-14)


def test_two_qubit_rotations_from_textbook_pauli_products():
    # Paulis written out here (not the oracle's tables); first wire = left factor
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    XX, YY, ZZ = np.kron(X, X), np.kron(Y, Y), np.kron(Z, Z)
    for t in (0.35, -1.4, 2.9):
        for name, H in (("IsingXX", -0.5 * XX), ("IsingYY", -0.5 * YY), ("IsingZZ", -0.5 * ZZ),
                        ("IsingXY", 0.25 * (XX + YY))):
            np.testing.assert_allclose(oracle.gate_matrix(name, [t]), scipy.linalg.expm(1j * t * H), atol=1e-14,
                                       err_msg=name)
        # controlled rotations: |1><1| (x) R on the target, identity where the control is 0
        out = oracle.apply_op(np.eye(4, dtype=np.complex128)[:, 1].copy(), Op("RY", (1,), (0,), controls=(0,)),
                              np.array([t]))
        np.testing.assert_allclose(out, [0, 1, 0, 0], atol=1e-15)  # |01>: control 0, untouched
        out = oracle.apply_op(np.eye(4, dtype=np.complex128)[:, 2].copy(), Op("RY", (1,), (0,), controls=(0,)),
                              np.array([t]))
        np.testing.assert_allclose(out, [0, 0, math.cos(t / 2), math.sin(t / 2)], atol=1e-15)


def test_rot_closed_form():
    for (phi, th, om) in [(0.1, 0.2, 0.3), (-1.0, 2.0, 4.0), (3.0, -0.7, 1.9)]:
        c, s = math.cos(th / 2), math.sin(th / 2)
        want = np.array([[cmath.exp(-0.5j * (phi + om)) * c, -cmath.exp(0.5j * (phi - om)) * s],
                         [cmath.exp(-0.5j * (phi - om)) * s, cmath.exp(0.5j * (phi + om)) * c]])
        np.testing.assert_allclose(oracle.gate_matrix("Rot", [phi, th, om]), want, atol=1e-14)


def test_givens_gates_rotate_only_inside_their_subspace():
    for t in (0.3, -1.7):
        M = oracle.gate_matrix("SingleExcitation", [t])
        sub = M[np.ix_([1, 2], [1, 2])]
        np.testing.assert_allclose(sub, [[math.cos(t / 2), -math.sin(t / 2)], [math.sin(t / 2), math.cos(t / 2)]])
        rest = [0, 3]
        np.testing.assert_allclose(M[np.ix_(rest, rest)], np.eye(2))
        D = oracle.gate_matrix("DoubleExcitation", [t])
        np.testing.assert_allclose(D[np.ix_([3, 12], [3, 12])],
                                   [[math.cos(t / 2), -math.sin(t / 2)], [math.sin(t / 2), math.cos(t / 2)]])
        others = [i for i in range(16) if i not in (3, 12)]
        np.testing.assert_allclose(D[np.ix_(others, others)], np.eye(14))


def _listing1_rows():
    rows = []
    for ln in open(os.path.join(GOLDEN, "listing1_semantics.txt")):
        if ln.strip() and not ln.startswith("#"):
            rows.append(ln.split())
    return rows


@pytest.mark.parametrize("n", [1, 3, 5])
def test_listing1_pauli_x_and_phase_shift_semantics(n):
    angle = 0.83
    for gate, inv, new0, new1 in _listing1_rows():
        for q in range(n):
            psi = random_state(n, 11 * n + q)
            out = psi.copy()
            op = Op(gate, (q,), (0,) if gate == "PhaseShift" else (), adjoint=bool(int(inv)))
            oracle.apply_op(out, op, np.array([angle]))
            for i0, i1 in enumeration.single_qubit_pairs(n, q):
                env = {"a0": psi[i0], "a1": psi[i1], "exp": cmath.exp, "i": 1j, "angle": angle}
                assert abs(out[i0] - eval(new0, env)) < 1e-15
                assert abs(out[i1] - eval(new1, env)) < 1e-15


# ---------------------------------------------------------------------------
# C loops vs dense reference; invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2), (5, 3), (6, 4), (7, 5)])
def test_oracle_forward_matches_dense_kronecker(n, seed):
    c, p = random_circuit(n, 25, seed, max_controls=2)
    psi0 = random_state(n, seed + 50)
    got = oracle.forward(c, p, psi0)
    want = dense.circuit_unitary(c, p) @ psi0
    np.testing.assert_allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("name", [g for g in GATE_ARITY if g != "Identity"])
def test_gate_then_inverse_is_identity_and_norm_preserved(name):
    n = 5
    k = GATE_ARITY[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    for trial in range(4):
        wires = tuple(int(w) for w in rng.permutation(n)[:k])
        free = [w for w in range(n) if w not in wires]
        controls = tuple(free[:trial % 2])
        op = Op(name, wires, tuple(range(GATE_NPARAMS[name])), controls)
        params = rng.uniform(-4, 4, size=GATE_NPARAMS[name])
        psi = random_state(n, trial)
        out = oracle.apply_op(psi.copy(), op, params)
        assert abs(oracle.norm2(out) - 1.0) < 1e-14
        back = oracle.apply_op(out, op, params, dagger=True)
        np.testing.assert_allclose(back, psi, atol=1e-14)


@pytest.mark.parametrize("n", range(1, 11))
def test_ghz_amplitudes(n):
    ops = [Op("Hadamard", (0,))] + [Op("PauliX", (i + 1,), controls=(i,)) for i in range(n - 1)]
    psi = oracle.forward(Circuit(n, ops, 0), np.zeros(0))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.abs(psi - want).max() < 1e-15
    assert np.count_nonzero(psi) == 2


@pytest.mark.parametrize("theta", [0.0, 0.37, 1.2, -2.5, math.pi])
def test_rx_expectations_closed_form(theta):
    c = Circuit(1, [Op("RX", (0,), (0,))], 1,
                [[Term(1.0, ((0, "Z"),))], [Term(1.0, ((0, "Y"),))], [Term(1.0, ((0, "X"),))]])
    psi = oracle.forward(c, np.array([theta]))
    E = oracle.expvals(psi, c.observables)
    assert abs(E[0] - math.cos(theta)) < 1e-15
    assert abs(E[1] + math.sin(theta)) < 1e-15
    assert abs(E[2]) < 1e-15
    _, J = oracle.adjoint_jacobian(c, np.array([theta]))
    assert abs(J[0, 0] + math.sin(theta)) < 1e-15     # d<Z>/dtheta = -sin(theta)


def _closed_form_pauli(n, paulis, psi):
    """P|i> = i^{nY} (-1)^{popcount(i & z)} |i ^ x> with bit (n-1-w) for wire w."""
    x = z = 0
    for w, l in paulis:
        b = 1 << (n - 1 - w)
        if l in "XY":
            x |= b
        if l in "YZ":
            z |= b
    ny = bin(x & z).count("1")
    out = np.zeros_like(psi)
    for i in range(1 << n):
        out[i ^ x] += (1j ** ny) * (-1) ** bin(i & z).count("1") * psi[i]
    return out


def test_pauli_words_closed_form_all_3q_words():
    n = 3
    psi = random_state(n, 5)
    for letters in itertools.product("IXYZ", repeat=n):
        paulis = tuple((w, l) for w, l in enumerate(letters) if l != "I")
        a = oracle.apply_pauli_word(psi, paulis)
        b = dense.pauli_word(n, paulis) @ psi
        c = _closed_form_pauli(n, paulis, psi)
        np.testing.assert_allclose(a, b, atol=1e-15)
        np.testing.assert_allclose(a, c, atol=1e-15)


def test_ry_product_state_closed_form():
    n, layers = 6, 3
    rng = np.random.default_rng(9)
    ops, p = [], 0
    for _ in range(layers):
        for w in range(n):
            ops.append(Op("RY", (w,), (p,)))
            p += 1
    params = rng.uniform(0, 2 * math.pi, size=p)
    obs = [[Term(1.0, ((w, "Z"),))] for w in range(n)]
    c = Circuit(n, ops, p, obs)
    E = oracle.expvals(oracle.forward(c, params), obs)
    for w in range(n):
        tot = sum(params[l * n + w] for l in range(layers))
        assert abs(E[w] - math.cos(tot)) < 1e-14


def test_hartree_fock_energy_closed_form():
    c, p = vqe_givens(n=10, electrons=4, n_singles=3, n_doubles=3, n_terms=60, seed=4)
    H = c.observables[0]
    psi = oracle.forward(c, np.zeros_like(p))          # zero angles: HF state untouched
    want = 0.0
    for t in H:
        if all(l == "Z" for _, l in t.paulis):
            occ = sum(1 for w, _ in t.paulis if (c.basis_state >> (c.n - 1 - w)) & 1)
            want += t.coeff * (-1) ** occ
    assert abs(oracle.expval(psi, H) - want) < 1e-13


def test_givens_circuit_preserves_hamming_weight():
    c, p = vqe_givens(n=10, electrons=4, n_singles=6, n_doubles=8, n_terms=5, seed=1)
    psi = oracle.forward(c, p * 10)
    for i in range(1 << c.n):
        if bin(i).count("1") != 4:
            assert psi[i] == 0.0


def test_oracle_reductions_do_not_depend_on_thread_count():
    a, b = random_state(15, 1), random_state(15, 2)
    t0 = oracle.num_threads()
    r_many = oracle.inner(a, b)
    oracle.set_num_threads(1)
    r_one = oracle.inner(a, b)
    oracle.set_num_threads(t0)
    assert r_many == r_one
    np.testing.assert_allclose(r_one, np.vdot(a, b), rtol=1e-13)


# ---------------------------------------------------------------------------
# Gradients
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,seed", [(2, 10), (3, 11), (4, 12), (5, 13), (6, 14)])
def test_adjoint_matches_dense_exact_derivative(n, seed):
    c, p = random_circuit(n, 18, seed, shared_params=True)
    rng = np.random.default_rng(seed)
    obs = [random_hamiltonian(n, 4, rng, weights=(1, 2)), random_hamiltonian(n, 3, rng, weights=(1, 2, 3))]
    E, J = oracle.adjoint_jacobian(c, p, obs)
    np.testing.assert_allclose(E, dense.expvals(c, p, obs), atol=1e-13)
    np.testing.assert_allclose(J, dense.exact_jacobian(c, p, obs), atol=1e-12)


@pytest.mark.parametrize("maker", ["layered", "sel", "qaoa", "rycz"])
def test_adjoint_matches_parameter_shift(maker):
    if maker == "layered":
        c, p = layered_circuit(5, 2, seed=1)
    elif maker == "sel":
        c, p = strongly_entangling(5, 2, seed=2)
    elif maker == "qaoa":
        c = qaoa_maxcut(6, 2, seed=3)
        p = np.random.default_rng(3).uniform(0, math.pi, size=4)
    else:
        c, p = ry_cz_brick(6, 3, seed=4)
    E, J = oracle.adjoint_jacobian(c, p)
    Jps = oracle.param_shift_jacobian(c, p)
    np.testing.assert_allclose(J, Jps, atol=1e-12)


@pytest.mark.parametrize("maker", ["layered", "sel", "qaoa", "vqe", "rycz"])
def test_workload_miniatures_match_the_dense_reference(maker):
    # each benchmark workload's own generator at a size the Kronecker reference
    # can hold: forward amplitudes, expectation values and the exact Jacobian
    # (dU/dtheta = i s G U), which also covers the Givens gates that the
    # two-term shift rule cannot
    if maker == "layered":
        c, p = layered_circuit(6, 3, seed=11)
    elif maker == "sel":
        c, p = strongly_entangling(6, 6, seed=12)  # CNOT ranges 1..5 (l mod 5 + 1)
    elif maker == "qaoa":
        c = qaoa_maxcut(6, 2, seed=13)
        p = np.random.default_rng(13).uniform(0, math.pi, size=4)
    elif maker == "vqe":
        c, p = vqe_givens(8, 4, 3, 4, 20, seed=14)
        p = p + np.random.default_rng(14).normal(0.0, 0.5, size=p.size)  # away from the HF point
    else:
        c, p = ry_cz_brick(8, 4, seed=15, dense_every=0)
    psi0 = dense.initial(c)
    np.testing.assert_allclose(oracle.forward(c, p, psi0), dense.state(c, p), atol=1e-13)
    E, J = oracle.adjoint_jacobian(c, p)
    np.testing.assert_allclose(E, dense.expvals(c, p), atol=1e-13)
    np.testing.assert_allclose(J, dense.exact_jacobian(c, p), atol=1e-12)
    assert np.abs(J).max() > 1e-3  # a nontrivial gradient


def test_adjoint_matches_finite_differences():
    c, p = random_circuit(4, 14, 77)
    obs = [[Term(0.7, ((0, "Z"), (2, "X"))), Term(-1.1, ((1, "Y"),))]]
    _, J = oracle.adjoint_jacobian(c, p, obs)
    Jfd = oracle.finite_diff_jacobian(c, p, obs)
    np.testing.assert_allclose(J, Jfd, atol=1e-7)


# ---------------------------------------------------------------------------
# Dense blocks (QubitUnitary) on the tape
# ---------------------------------------------------------------------------
CNOT_TEXTBOOK = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)


@pytest.mark.parametrize("wires", [(0, 1), (1, 0), (2, 0), (1, 3)])
def test_dense_block_wire_order_is_the_textbook_cnot(wires):
    # the textbook CNOT matrix (first wire = control = most significant bit) on
    # `wires` must equal the base gate PauliX on wires[1] controlled by wires[0]
    n = 4
    psi0 = random_state(n, 31)
    a = oracle.copy(psi0)
    oracle.apply_op(a, MatrixOp(wires, CNOT_TEXTBOOK), np.zeros(0))
    b = oracle.copy(psi0)
    oracle.apply_op(b, Op("PauliX", (wires[1],), controls=(wires[0],)), np.zeros(0))
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("wires,controls", [((5, 0, 3, 1, 4), ()), ((0, 1, 2, 3, 4), ()), ((4, 2, 0, 5, 1), (3,))])
def test_dense_block_forward_matches_dense_kronecker(wires, controls):
    n = 6
    rng = np.random.default_rng(41)
    ops = [Op("RY", (w,), (w,)) for w in range(n)]
    ops += [MatrixOp(wires, random_unitary(5, rng), controls)]
    ops += [Op("RX", (w,), (n + w,)) for w in range(n)]
    ops += [MatrixOp(wires, random_unitary(5, rng), controls, adjoint=True)]
    c = Circuit(n, ops, 2 * n, [])
    p = rng.uniform(0, 2 * math.pi, 2 * n)
    np.testing.assert_allclose(oracle.forward(c, p), dense.state(c, p), atol=1e-13)


def test_dense_block_adjoint_flag_is_the_conjugate_transpose():
    n = 7
    U = random_unitary(5, np.random.default_rng(43))
    psi0 = random_state(n, 43)
    a = oracle.copy(psi0)
    oracle.apply_op(a, MatrixOp((6, 2, 4, 0, 3), U, adjoint=True), np.zeros(0))
    b = oracle.copy(psi0)
    oracle.apply_op(b, MatrixOp((6, 2, 4, 0, 3), U.conj().T.copy()), np.zeros(0))
    np.testing.assert_array_equal(a, b)
    oracle.apply_op(a, MatrixOp((6, 2, 4, 0, 3), U), np.zeros(0))  # U U^dagger = I
    np.testing.assert_allclose(a, psi0, atol=1e-14)


def test_rycz_dense_block_windows_are_distinct_wires_and_touch_bit0():
    for n in (10, 12, 30):
        ws = [dense_block_wires(n, b) for b in range(4)]
        assert all(len(set(w)) == 5 and min(w) >= 0 and max(w) < n for w in ws)
        assert any(n - 1 in w for w in ws)  # wire n-1 = global index bit 0


def test_adjoint_through_dense_blocks_matches_parameter_shift():
    # RY + CZ brick with a dense block after every second layer (all four windows)
    c, p = ry_cz_brick(10, 8, seed=4, dense_every=2)
    assert sum(op.name == "QubitUnitary" for op in c.ops) == 4
    E, J = oracle.adjoint_jacobian(c, p)
    Jps = oracle.param_shift_jacobian(c, p)
    np.testing.assert_allclose(J, Jps, atol=1e-12)
    np.testing.assert_allclose(E, oracle.expvals(oracle.forward(c, p), c.observables), atol=1e-14)


def test_adjoint_through_a_controlled_dense_block_matches_the_exact_derivative():
    n = 6
    rng = np.random.default_rng(47)
    ops = [Op("RX", (w,), (w,)) for w in range(n)]
    ops += [MatrixOp((0, 2, 4, 5, 1), random_unitary(5, rng), (3,), (0,))]
    ops += [Op("RY", (w,), (n + w,)) for w in range(n)]
    obs = [[Term(1.0, ((2, "Z"),))], [Term(0.4, ((0, "X"), (5, "Y")))]]
    c = Circuit(n, ops, 2 * n, obs)
    p = rng.uniform(0, 2 * math.pi, 2 * n)
    _, J = oracle.adjoint_jacobian(c, p)
    np.testing.assert_allclose(J, dense.exact_jacobian(c, p), atol=1e-12)


# ---------------------------------------------------------------------------
# Observables given as Hermitian matrices
# ---------------------------------------------------------------------------
def _random_hermitian(k, rng):
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    return (a + a.conj().T) / 2


@pytest.mark.parametrize("theta", [0.0, 0.4, 2.2, -1.3])
def test_matrix_observable_projector_after_rx_closed_form(theta):
    # |1><1| on wire 1 after RX(theta) there: probability sin^2(theta / 2)
    c = Circuit(3, [Op("RX", (1,), (0,))], 1, [])
    psi = oracle.forward(c, np.array([theta]))
    proj = oracle.MatrixObservable([1], np.diag([0.0, 1.0]))
    assert oracle.expval(psi, proj) == pytest.approx(math.sin(theta / 2) ** 2, abs=1e-15)


def test_matrix_observable_of_a_pauli_word_equals_the_pauli_path():
    # the Kronecker matrix of X (x) Y (x) Z on wires (4, 0, 2) against the
    # per-wire Pauli application of the same word
    n = 5
    psi = random_state(n, 61)
    m = np.kron(np.kron(oracle.PAULI["X"], oracle.PAULI["Y"]), oracle.PAULI["Z"])
    word = [Term(1.0, ((4, "X"), (0, "Y"), (2, "Z")))]
    got = oracle.expval(psi, oracle.MatrixObservable([4, 0, 2], m))
    assert got == pytest.approx(oracle.expval(psi, word), abs=1e-14)
    np.testing.assert_allclose(oracle.MatrixObservable([4, 0, 2], m).apply(psi),
                               oracle.apply_hamiltonian(psi, word), atol=1e-15)


def test_matrix_observable_expval_and_variance_match_dense_algebra():
    n = 5
    rng = np.random.default_rng(62)
    A = _random_hermitian(3, rng)
    wires = [3, 1, 4]
    psi = random_state(n, 62)
    full = dense.embed(n, wires, A)
    obs = oracle.MatrixObservable(wires, A)
    e = np.vdot(psi, full @ psi).real
    assert oracle.expval(psi, obs) == pytest.approx(e, abs=1e-13)
    assert oracle.variance(psi, obs) == pytest.approx(np.vdot(psi, full @ full @ psi).real - e * e, abs=1e-12)


def test_adjoint_with_a_matrix_observable_matches_parameter_shift():
    c, p = layered_circuit(5, 2, seed=63)
    A = _random_hermitian(2, np.random.default_rng(63))
    obs = [oracle.MatrixObservable([2, 0], A)]
    _, J = oracle.adjoint_jacobian(c, p, obs)
    np.testing.assert_allclose(J, oracle.param_shift_jacobian(c, p, obs), atol=1e-12)


def test_vjp_is_gradient_weighted_jacobian_rows():
    c, p = strongly_entangling(4, 2, seed=5)
    g = np.random.default_rng(1).normal(size=len(c.observables))
    _, J = oracle.adjoint_jacobian(c, p)
    np.testing.assert_allclose(oracle.adjoint_vjp(c, p, g), g @ J, atol=1e-13)


def _qaoa_p1_zz(gamma, beta, du, dv, f):
    """<Z_u Z_v> after H^n, exp(-i gamma Z_aZ_b) per edge, exp(-i beta X) per wire.

    From the p=1 MaxCut edge expectation of Wang, Hadfield, Jiang and Rieffel
    (2018) for e^{-i g C} e^{-i b B} with C_uv = (1 - Z_uZ_v)/2; this circuit
    is g = -2 gamma, b = beta.  du, dv = degree - 1; f = triangles on the edge.
    """
    g = -2.0 * gamma
    b = beta
    cuv = (0.5 + 0.25 * math.sin(4 * b) * math.sin(g) * (math.cos(g) ** du + math.cos(g) ** dv)
           - 0.25 * math.sin(2 * b) ** 2 * math.cos(g) ** (du + dv - 2 * f) * (1 - math.cos(2 * g) ** f))
    return 1.0 - 2.0 * cuv


def test_single_edge_qaoa_by_hand():
    # Heisenberg picture by hand: Z -> cos(2b) Z + sin(2b) Y per wire, so
    # <Z0Z1> = 2 sin(2b)cos(2b) sin(2 gamma) = sin(4b) sin(2 gamma).
    for gm, bt in [(0.3, 0.2), (1.1, 2.0), (2.9, 0.7)]:
        c = qaoa_maxcut(2, 1, edges=[(0, 1)])
        E = oracle.expvals(oracle.forward(c, np.array([gm, bt])), c.observables)
        assert abs(E[0] - math.sin(4 * bt) * math.sin(2 * gm)) < 1e-14
        assert abs(_qaoa_p1_zz(gm, bt, 0, 0, 0) - math.sin(4 * bt) * math.sin(2 * gm)) < 1e-14


@pytest.mark.parametrize("n", [8, 10])
def test_qaoa_p1_closed_form_on_regular_graphs(n):
    rng = np.random.default_rng(n)
    edges = regular_graph(n, rng)
    adj = {v: set() for v in range(n)}
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    for gm, bt in [(0.4, 0.3), (1.7, 2.2)]:
        c = qaoa_maxcut(n, 1, edges=edges)
        psi = oracle.forward(c, np.array([gm, bt]))
        for (u, v) in edges:
            e = oracle.expval(psi, [Term(1.0, ((u, "Z"), (v, "Z")))])
            f = len(adj[u] & adj[v])
            want = _qaoa_p1_zz(gm, bt, len(adj[u]) - 1, len(adj[v]) - 1, f)
            assert abs(e - want) < 1e-13


# ---- variance: closed forms, eigenstates, dense reference -------------------
def test_variance_after_rx_closed_form():
    # RX(t)|0> = cos(t/2)|0> - i sin(t/2)|1>: <Z> = cos t, <Y> = -sin t, <X> = 0,
    # and every Pauli word squares to I, so Var(P) = 1 - <P>^2.
    for t in (0.0, 0.37, 1.9, 3.0):
        psi = oracle.forward(Circuit(1, [Op("RX", (0,), (0,))], 1, []), np.array([t]))
        assert abs(oracle.variance(psi, [Term(1.0, ((0, "Z"),))]) - math.sin(t) ** 2) < 1e-14
        assert abs(oracle.variance(psi, [Term(1.0, ((0, "Y"),))]) - math.cos(t) ** 2) < 1e-14
        assert abs(oracle.variance(psi, [Term(1.0, ((0, "X"),))]) - 1.0) < 1e-14
        # Var(a Z + b) = a^2 Var(Z): the identity term only shifts
        v = oracle.variance(psi, [Term(-2.5, ((0, "Z"),)), Term(0.75, ())])
        assert abs(v - 6.25 * math.sin(t) ** 2) < 1e-13


def test_variance_vanishes_on_eigenstates():
    n = 4
    ops = [Op("Hadamard", (0,))] + [Op("PauliX", (w + 1,), controls=(w,)) for w in range(n - 1)]
    psi = oracle.forward(Circuit(n, ops, 0, []), np.zeros(0))  # GHZ: eigenstate of Z_i Z_j and X^n
    H = [Term(0.7, ((0, "Z"), (3, "Z"))), Term(-1.3, ((0, "X"), (1, "X"), (2, "X"), (3, "X")))]
    assert abs(oracle.variance(psi, H)) < 1e-13
    assert abs(oracle.expval(psi, H) - (0.7 - 1.3)) < 1e-13


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_variance_matches_dense_hamiltonian(seed):
    n = 5
    rng = np.random.default_rng(seed)
    psi = random_state(n, seed)
    H = random_hamiltonian(n, 12, rng, weights=(1, 2, 3))
    Hd = dense.hamiltonian(n, H)
    e = np.vdot(psi, Hd @ psi).real
    want = np.vdot(psi, Hd @ (Hd @ psi)).real - e * e
    assert abs(oracle.variance(psi, H) - want) < 1e-12 * max(1.0, abs(want))


# ---- probabilities and samples ----------------------------------------------
def test_probabilities_of_a_product_state_closed_form():
    th = np.array([0.3, 1.1, 2.5, 0.9])
    c = Circuit(4, [Op("RY", (w,), (w,)) for w in range(4)], 4, [])
    psi = oracle.forward(c, th)
    for w in range(4):
        p = oracle.probabilities(psi, [w])
        assert abs(p[1] - math.sin(th[w] / 2) ** 2) < 1e-15 and abs(p.sum() - 1) < 1e-15
    p = oracle.probabilities(psi, [3, 1])  # wires[0] is the most significant outcome bit
    for b3 in (0, 1):
        for b1 in (0, 1):
            want = ((math.sin(th[3] / 2) ** 2) if b3 else (math.cos(th[3] / 2) ** 2)) * \
                   ((math.sin(th[1] / 2) ** 2) if b1 else (math.cos(th[1] / 2) ** 2))
            assert abs(p[2 * b3 + b1] - want) < 1e-15


def test_probabilities_brute_force_and_wire_order():
    n = 4
    psi = random_state(n, 5)
    for wires in ([0], [3], [2, 0], [1, 3, 2], [0, 1, 2, 3], []):
        want = np.zeros(1 << len(wires))
        for i in range(1 << n):
            bits = [(i >> (n - 1 - w)) & 1 for w in wires]
            b = 0
            for x in bits:
                b = 2 * b + x
            want[b] += abs(psi[i]) ** 2
        assert np.abs(oracle.probabilities(psi, wires) - want).max() < 1e-15
    # a basis state |i> is one-hot on its own bits
    e = oracle.basis_state(n, 0b1011)
    assert list(oracle.probabilities(e, [2, 0])) == [0.0, 0.0, 0.0, 1.0]


def test_sampling_by_inverse_transform():
    n = 3
    ghz = oracle.forward(Circuit(n, [Op("Hadamard", (0,))] + [Op("PauliX", (w + 1,), controls=(w,))
                                                              for w in range(n - 1)], 0, []), np.zeros(0))
    u = np.array([0.0, 0.2, 0.4999999, 0.5, 0.75, 0.9999999])
    assert list(oracle.sample(ghz, [0, 1, 2], u)) == [0, 0, 0, 7, 7, 7]
    assert list(oracle.sample(oracle.basis_state(n, 5), [0, 1, 2], u)) == [5] * 6
    # empirical frequencies of seeded uniforms: within 5 sigma of the probabilities
    psi = random_state(n, 9)
    p = oracle.probabilities(psi, [2, 0])
    shots = 20000
    s = oracle.sample(psi, [2, 0], np.random.default_rng(9).random(shots))
    freq = np.bincount(s.astype(np.int64), minlength=4) / shots
    assert np.all(np.abs(freq - p) <= 5 * np.sqrt(p * (1 - p) / shots) + 1e-12)


def test_sampling_stratified_uniforms_give_exact_counts():
    # K evenly spaced uniforms (k + 1/2) / K: outcome b takes the grid points in
    # [CDF_{b-1}, CDF_b), i.e. K p_b of them up to one at each end
    psi = random_state(5, 21)
    for wires in ([1, 4], [0, 2, 3], [4]):
        p = oracle.probabilities(psi, wires)
        K = 100003
        s = oracle.sample(psi, wires, (np.arange(K) + 0.5) / K)
        counts = np.bincount(s.astype(np.int64), minlength=p.size)
        assert counts.sum() == K and np.all(np.abs(counts - K * p) <= 1.0 + 1e-9)
        assert np.all(np.diff(s.astype(np.int64)) >= 0)  # monotone in u


def test_probabilities_agree_with_z_expectations():
    # <Z_w> = p_w(0) - p_w(1), and <Z_a Z_b> = sum_b (-1)^(b_a + b_b) p_ab(b):
    # the marginal sums against the Pauli-word path
    n = 5
    psi = random_state(n, 22)
    for w in range(n):
        p = oracle.probabilities(psi, [w])
        assert abs(oracle.expval(psi, [Term(1.0, ((w, "Z"),))]) - (p[0] - p[1])) < 1e-14
    for a, b in ((0, 4), (3, 1), (2, 3)):
        p = oracle.probabilities(psi, [a, b])
        want = p[0] - p[1] - p[2] + p[3]
        assert abs(oracle.expval(psi, [Term(1.0, ((a, "Z"), (b, "Z")))]) - want) < 1e-14


# ---- forward-mode Jacobian-vector product -----------------------------------
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_jvp_matches_dense_exact_jacobian(seed):
    n = 4
    c, p = random_circuit(n, 30, seed, max_controls=1, shared_params=(seed == 2))
    rng = np.random.default_rng(seed)
    obs = [random_hamiltonian(n, 6, rng, weights=(1, 2)) for _ in range(3)]
    v = rng.normal(size=c.n_params)
    want = dense.exact_jacobian(c, p, obs) @ v
    assert np.abs(oracle.jvp(c, p, v, obs) - want).max() < 1e-11


def test_jvp_matches_central_differences_along_the_tangent():
    c, p = layered_circuit(4, 3, seed=5)
    v = np.random.default_rng(5).normal(size=c.n_params)
    h = 1e-5
    ep = oracle.expvals(oracle.forward(c, p + h * v), c.observables)
    em = oracle.expvals(oracle.forward(c, p - h * v), c.observables)
    assert np.abs(oracle.jvp(c, p, v) - (ep - em) / (2 * h)).max() < 1e-7


def test_jvp_of_unit_tangents_is_the_parameter_shift_column():
    c, p = layered_circuit(3, 2, seed=6)
    Js = oracle.param_shift_jacobian(c, p)
    for q in (0, 5, c.n_params - 1):
        e = np.zeros(c.n_params)
        e[q] = 1.0
        assert np.abs(oracle.jvp(c, p, e) - Js[:, q]).max() < 1e-12


# ---- sparse observables --------------------------------------------------------
def _csr_of(M):
    rows, cols = np.nonzero(M)
    indptr = np.zeros(M.shape[0] + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    return oracle.CSRObservable(np.cumsum(indptr), cols, M[rows, cols])


def test_sparse_observable_equals_its_pauli_sum():
    n = 5
    rng = np.random.default_rng(11)
    H = random_hamiltonian(n, 9, rng, weights=(1, 2, 3))
    Hs = _csr_of(dense.hamiltonian(n, H))
    psi = random_state(n, 11)
    assert abs(oracle.expval(psi, Hs) - oracle.expval(psi, H)) < 1e-13
    c, p = random_circuit(n, 25, 11, max_controls=1)
    E1, J1 = oracle.adjoint_jacobian(c, p, [H])
    E2, J2 = oracle.adjoint_jacobian(c, p, [Hs])
    assert abs(E1[0] - E2[0]) < 1e-13 and np.abs(J1 - J2).max() < 1e-12


def test_sparse_observable_matches_dense_algebra():
    n = 5
    rng = np.random.default_rng(12)
    A = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for _ in range(60):  # random sparse Hermitian
        i, j = rng.integers(0, 1 << n, 2)
        z = rng.normal() + 1j * rng.normal()
        A[i, j] += z
        A[j, i] += np.conj(z)
    Hs = _csr_of(A)
    psi = random_state(n, 12)
    assert np.abs(Hs.apply(psi) - A @ psi).max() < 1e-13
    assert abs(oracle.expval(psi, Hs) - np.vdot(psi, A @ psi).real) < 1e-12
    c, p = random_circuit(n, 20, 12)
    J = oracle.adjoint_jacobian(c, p, [Hs])[1]
    # central differences of <psi|A|psi> (sanity bar; the exact pin is the Pauli-sum test above)
    Jd = np.zeros((1, c.n_params))
    h = 1e-6
    for q in range(c.n_params):
        e = np.zeros(c.n_params)
        e[q] = h
        fp = np.vdot(oracle.forward(c, p + e), A @ oracle.forward(c, p + e)).real
        fm = np.vdot(oracle.forward(c, p - e), A @ oracle.forward(c, p - e)).real
        Jd[0, q] = (fp - fm) / (2 * h)
    assert np.abs(J - Jd).max() < 1e-6 * max(1.0, np.abs(Jd).max())
