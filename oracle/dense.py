"""Dense Kronecker-product reference for small circuits (n <= 8).

TEST INFRASTRUCTURE ONLY.  Independent of the C loops in ``sv_oracle.c``: every
operator is built as a full 2^n x 2^n matrix from ``np.kron`` of single-wire
factors, with wire 0 the leftmost factor (the most significant index bit,
Alg. 1).  It pins the oracle's gate application, Pauli expectation values and
adjoint Jacobian:

* U_total = prod_k (operator of op k),
* dU_k/dtheta = i s G_k U_k exactly (U = exp(i s theta G)),
* dE/dparam = sum over uses of 2 Re <psi| O | U_N..U_{k+1} dU_k U_{k-1}..U_1 psi0>.
"""

from __future__ import annotations

from functools import reduce
from typing import Sequence

import numpy as np

from .core import PAULI, generator, op_angles, gate_matrix, expand, _step_matrix

I2 = np.eye(2, dtype=np.complex128)


def _ket_bra(a: int, b: int) -> np.ndarray:
    m = np.zeros((2, 2), dtype=np.complex128)
    m[a, b] = 1.0
    return m


def embed(n: int, wires: Sequence[int], M: np.ndarray) -> np.ndarray:
    """Full operator of the local matrix M on ``wires``: sum_ab M_ab (x)_j |a_j><b_j|."""
    k = len(wires)
    full = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for a in range(1 << k):
        for b in range(1 << k):
            if M[a, b] == 0:
                continue
            factors = [I2] * n
            for j, w in enumerate(wires):
                factors[w] = _ket_bra((a >> (k - 1 - j)) & 1, (b >> (k - 1 - j)) & 1)
            full += M[a, b] * reduce(np.kron, factors)
    return full


def control_projector(n: int, controls: Sequence[int], values: Sequence[int]) -> np.ndarray:
    factors = [I2] * n
    for c, v in zip(controls, values):
        factors[c] = _ket_bra(v, v)
    return reduce(np.kron, factors)


def controlled(n: int, wires, M, controls, values) -> np.ndarray:
    """I + P_c ((M on wires) - I): M acts only where the controls hold ``values``."""
    U = embed(n, wires, M)
    if not controls:
        return U
    P = control_projector(n, controls, values)
    eye = np.eye(1 << n, dtype=np.complex128)
    return eye + P @ (U - eye)


def op_unitary(n: int, op, params) -> np.ndarray:
    if op.name == "QubitUnitary":
        M = np.array(op.matrix, dtype=np.complex128)
    else:
        M = gate_matrix(op.name, op_angles(op, params))
    if op.adjoint:
        M = M.conj().T
    return controlled(n, op.wires, M, op.controls, op.ctrl_values)


def circuit_unitary(circuit, params) -> np.ndarray:
    U = np.eye(1 << circuit.n, dtype=np.complex128)
    for op in circuit.ops:
        U = op_unitary(circuit.n, op, params) @ U
    return U


def initial(circuit) -> np.ndarray:
    v = np.zeros(1 << circuit.n, dtype=np.complex128)
    v[circuit.basis_state] = 1.0
    return v


def state(circuit, params) -> np.ndarray:
    return circuit_unitary(circuit, params) @ initial(circuit)


def pauli_word(n: int, paulis) -> np.ndarray:
    factors = [I2] * n
    for w, letter in paulis:
        factors[w] = PAULI[letter]
    return reduce(np.kron, factors)


def hamiltonian(n: int, terms) -> np.ndarray:
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t in terms:
        H += t.coeff * pauli_word(n, t.paulis)
    return H


def expvals(circuit, params, observables=None) -> np.ndarray:
    obs = circuit.observables if observables is None else observables
    psi = state(circuit, params)
    return np.array([np.vdot(psi, hamiltonian(circuit.n, H) @ psi).real for H in obs])


def exact_jacobian(circuit, params, observables=None) -> np.ndarray:
    """J[j, p] from dU/dtheta = i s G U for every angle use (Rot expanded)."""
    n = circuit.n
    obs = circuit.observables if observables is None else observables
    Hs = [hamiltonian(n, H) for H in obs]
    steps = expand(circuit.ops)
    mats = []
    for st in steps:
        M = _step_matrix(st, params)
        mats.append(controlled(n, st.wires, M, st.controls, st.cvals))
    psi0 = initial(circuit)
    # prefix states and suffix products
    prefix = [psi0]
    for U in mats:
        prefix.append(U @ prefix[-1])
    psi = prefix[-1]
    J = np.zeros((len(obs), circuit.n_params))
    suffix = np.eye(1 << n, dtype=np.complex128)
    for k in range(len(steps) - 1, -1, -1):
        st = steps[k]
        if st.param is not None:
            G, s = generator(st.name)
            if st.adjoint:
                s = -s
            Gc = embed(n, st.wires, G)
            if st.controls:
                Gc = control_projector(n, st.controls, st.cvals) @ Gc
            dpsi = suffix @ (1j * s * Gc @ (mats[k] @ prefix[k]))
            for j, H in enumerate(Hs):
                J[j, st.param] += st.scale * 2.0 * np.vdot(psi, H @ dpsi).real
        suffix = suffix @ mats[k]
    return J
