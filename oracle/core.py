"""FP64 oracle: gates, Pauli sums, forward pass, adjoint Jacobian.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is computed, and where the paper fixes it:

* State: 2^n complex amplitudes, wire 0 = most significant index bit
  (Alg. 1: q_offset = n - q - 1).  Templated float/double in the paper
  (Sec. 2); here always complex128.
* Gates (Sec. 2.1.2 gate list; Listing 1; Eq. 1): every rotation is
  exp(-i theta P / 2); PhaseShift multiplies the |1> component by e^{i phi}
  and its inverse by e^{-i phi} (Listing 1); IsingXX is the printed matrix of
  Eq. 1 and IsingYY / IsingZZ follow the same form; IsingXY(theta) =
  exp(i theta/4 (XX + YY)); Rot(phi, theta, omega) = RZ(omega) RY(theta) RZ(phi);
  SingleExcitation / DoubleExcitation rotate by theta/2 inside
  {|01>, |10>} / {|0011>, |1100>} (Sec. 3.2) and are the identity elsewhere.
  The ``inverse`` flag of Listing 1 applies the conjugate transpose.
* Controlled gates act only where the control wires hold the prescribed
  values (Alg. 2, "all control bits equal to 1 (or a prescribed bit string)").
* Generators (Sec. 2.1.2, "the respective generators ... used for gradient
  evaluations"): U(theta) = exp(i s theta G).
* Observables (Sec. 2.2, Listing 2): Hamiltonians sum_t c_t P_t of Pauli
  words; a word is applied wire by wire with the 2x2 Pauli matrices.
* Adjoint Jacobian (the adjoint method the paper cites in Sec. 2.1 and 3.1.1):
  phi = final state, lambda_j = O_j phi; for ops in reverse order, if the op
  carries an angle, J[j, p] += scale * (-2 s) Im <lambda_j | G phi>; then
  phi <- U^dagger phi and lambda_j <- U^dagger lambda_j.  Multi-angle Rot is
  expanded into RZ, RY, RZ before the sweep.  The Jacobian of a Hamiltonian
  observable is one row for the whole sum (Listing 2).
"""

from __future__ import annotations

import ctypes
import math
import time
from typing import List, Sequence, Tuple

import numpy as np

from . import build as _build

# ---------------------------------------------------------------------------
# C loops
# ---------------------------------------------------------------------------
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_apply.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int, ip, ip]
        L.orc_apply.restype = ctypes.c_int
        L.orc_project_controls.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ip]
        L.orc_project_controls.restype = ctypes.c_int
        L.orc_inner.argtypes = [dp, dp, ctypes.c_int, dp]
        L.orc_inner.restype = None
        L.orc_axpy.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_axpy.restype = None
        L.orc_copy.argtypes = [dp, dp, ctypes.c_int]
        L.orc_copy.restype = None
        L.orc_basis.argtypes = [dp, ctypes.c_int, ctypes.c_int64]
        L.orc_basis.restype = None
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


def _dptr(a: np.ndarray):
    assert a.dtype in (np.complex128, np.float64) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iarr(xs: Sequence[int]):
    arr = (ctypes.c_int * max(1, len(xs)))(*[int(x) for x in xs])
    return arr


def _nqubits(psi: np.ndarray) -> int:
    n = int(round(math.log2(psi.size)))
    assert (1 << n) == psi.size
    return n


def apply_matrix(psi: np.ndarray, M: np.ndarray, wires: Sequence[int],
                 controls: Sequence[int] = (), control_values: Sequence[int] = ()) -> np.ndarray:
    """In place: apply the 2^k x 2^k matrix M to ``wires`` (wires[0] = local MSB)."""
    n = _nqubits(psi)
    k = len(wires)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    assert M.shape == (1 << k, 1 << k)
    cv = list(control_values) if control_values else [1] * len(controls)
    rc = lib().orc_apply(_dptr(psi), n, k, _iarr(wires), _dptr(M), len(controls),
                         _iarr(controls), _iarr(cv))
    if rc != 0:
        raise ValueError("orc_apply: bad arguments")
    return psi


def project_controls(psi: np.ndarray, controls: Sequence[int], control_values: Sequence[int]):
    n = _nqubits(psi)
    cv = list(control_values) if control_values else [1] * len(controls)
    if lib().orc_project_controls(_dptr(psi), n, len(controls), _iarr(controls), _iarr(cv)) != 0:
        raise ValueError("orc_project_controls: bad arguments")
    return psi


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """<a|b> = sum_i conj(a_i) b_i, fixed-order blocked FP64 sum."""
    out = np.zeros(2)
    lib().orc_inner(_dptr(a), _dptr(b), _nqubits(a), _dptr(out))
    return complex(out[0], out[1])


def axpy(y: np.ndarray, x: np.ndarray, c: complex) -> np.ndarray:
    lib().orc_axpy(_dptr(y), _dptr(x), _nqubits(y), float(np.real(c)), float(np.imag(c)))
    return y


def copy(x: np.ndarray) -> np.ndarray:
    y = np.empty_like(x)
    lib().orc_copy(_dptr(y), _dptr(x), _nqubits(x))
    return y


def basis_state(n: int, index: int = 0) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().orc_basis(_dptr(psi), n, int(index))
    return psi


# ---------------------------------------------------------------------------
# Gate matrices and generators
# ---------------------------------------------------------------------------
I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"X": PX, "Y": PY, "Z": PZ, "I": I2}


def _rot_half(theta: float) -> Tuple[float, float]:
    return math.cos(theta / 2.0), math.sin(theta / 2.0)


def gate_matrix(name: str, angles: Sequence[float] = ()) -> np.ndarray:
    """Matrix of a base gate in the local basis (first wire = most significant)."""
    a = [float(x) for x in angles]
    if name == "Identity":
        return I2.copy()
    if name == "PauliX":
        return PX.copy()
    if name == "PauliY":
        return PY.copy()
    if name == "PauliZ":
        return PZ.copy()
    if name == "Hadamard":
        return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    if name == "S":
        return np.diag([1.0, 1j]).astype(np.complex128)
    if name == "T":
        return np.diag([1.0, np.exp(1j * math.pi / 4)]).astype(np.complex128)
    if name == "PhaseShift":  # Listing 1: |1> component times e^{i phi}
        return np.diag([1.0, np.exp(1j * a[0])]).astype(np.complex128)
    if name == "RX":
        c, s = _rot_half(a[0])
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
    if name == "RY":
        c, s = _rot_half(a[0])
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if name == "RZ":
        return np.diag([np.exp(-0.5j * a[0]), np.exp(0.5j * a[0])]).astype(np.complex128)
    if name == "Rot":  # Rot(phi, theta, omega) = RZ(omega) RY(theta) RZ(phi)
        return gate_matrix("RZ", [a[2]]) @ gate_matrix("RY", [a[1]]) @ gate_matrix("RZ", [a[0]])
    if name == "SWAP":
        M = np.zeros((4, 4), dtype=np.complex128)
        M[0, 0] = M[1, 2] = M[2, 1] = M[3, 3] = 1.0
        return M
    if name == "IsingXX":  # Eq. 1
        c, s = _rot_half(a[0])
        M = np.zeros((4, 4), dtype=np.complex128)
        for i in range(4):
            M[i, i] = c
            M[i, 3 - i] = -1j * s
        return M
    if name == "IsingYY":  # exp(-i theta/2 Y(x)Y): corner entries flip sign w.r.t. Eq. 1
        c, s = _rot_half(a[0])
        M = np.zeros((4, 4), dtype=np.complex128)
        for i in range(4):
            M[i, i] = c
        M[0, 3] = M[3, 0] = 1j * s
        M[1, 2] = M[2, 1] = -1j * s
        return M
    if name == "IsingZZ":
        e = np.exp(-0.5j * a[0])
        return np.diag([e, np.conj(e), np.conj(e), e]).astype(np.complex128)
    if name == "IsingXY":  # exp(i theta/4 (XX + YY))
        c, s = _rot_half(a[0])
        M = np.eye(4, dtype=np.complex128)
        M[1, 1] = M[2, 2] = c
        M[1, 2] = M[2, 1] = 1j * s
        return M
    if name == "SingleExcitation":
        c, s = _rot_half(a[0])
        M = np.eye(4, dtype=np.complex128)
        M[1, 1] = M[2, 2] = c
        M[1, 2] = -s
        M[2, 1] = s
        return M
    if name == "DoubleExcitation":
        c, s = _rot_half(a[0])
        M = np.eye(16, dtype=np.complex128)
        M[3, 3] = M[12, 12] = c
        M[3, 12] = -s
        M[12, 3] = s
        return M
    raise ValueError(f"unknown gate {name}")


def generator(name: str) -> Tuple[np.ndarray, float]:
    """(G, s) with U(theta) = exp(i s theta G) for the one-angle gates."""
    if name == "RX":
        return PX.copy(), -0.5
    if name == "RY":
        return PY.copy(), -0.5
    if name == "RZ":
        return PZ.copy(), -0.5
    if name == "PhaseShift":
        return np.diag([0.0, 1.0]).astype(np.complex128), 1.0
    if name == "IsingXX":
        return np.kron(PX, PX), -0.5
    if name == "IsingYY":
        return np.kron(PY, PY), -0.5
    if name == "IsingZZ":
        return np.kron(PZ, PZ), -0.5
    if name == "IsingXY":
        return np.kron(PX, PX) + np.kron(PY, PY), 0.25
    if name == "SingleExcitation":
        G = np.zeros((4, 4), dtype=np.complex128)
        G[1, 2] = -1j
        G[2, 1] = 1j
        return G, -0.5
    if name == "DoubleExcitation":
        G = np.zeros((16, 16), dtype=np.complex128)
        G[3, 12] = -1j
        G[12, 3] = 1j
        return G, -0.5
    raise ValueError(f"{name} has no single generator")


def pauli_word_matrix(paulis, n_local_wires: Sequence[int]) -> np.ndarray:
    """Dense matrix of a Pauli word on the listed wires (helper for small tests)."""
    d = dict(paulis)
    M = np.ones((1, 1), dtype=np.complex128)
    for w in n_local_wires:
        M = np.kron(M, PAULI[d.get(w, "I")])
    return M


# ---------------------------------------------------------------------------
# Ops
# ---------------------------------------------------------------------------
def op_angles(op, params: np.ndarray) -> List[float]:
    return [op.scale * float(params[i]) for i in op.params]


def op_matrix(op, params: np.ndarray) -> np.ndarray:
    """Matrix of a base gate at its angles, or a QubitUnitary's own matrix;
    conjugate-transposed under the op's adjoint flag (Listing 1's inverse)."""
    if op.name == "QubitUnitary":
        M = np.array(op.matrix, dtype=np.complex128)
    else:
        M = gate_matrix(op.name, op_angles(op, params))
    return M.conj().T.copy() if op.adjoint else M


def apply_op(psi: np.ndarray, op, params: np.ndarray, dagger: bool = False) -> np.ndarray:
    """Apply op (or its conjugate transpose when ``dagger``) in place."""
    M = op_matrix(op, params)
    if dagger:
        M = M.conj().T.copy()
    return apply_matrix(psi, M, op.wires, op.controls, op.ctrl_values)


def initial_state(circuit) -> np.ndarray:
    return basis_state(circuit.n, circuit.basis_state)


def forward(circuit, params: np.ndarray, psi0: np.ndarray | None = None) -> np.ndarray:
    """psi = U_N ... U_1 |psi0> (default |basis_state> of the circuit)."""
    psi = initial_state(circuit) if psi0 is None else copy(np.ascontiguousarray(psi0, np.complex128))
    for op in circuit.ops:
        apply_op(psi, op, params)
    return psi


def apply_pauli_word(psi: np.ndarray, paulis) -> np.ndarray:
    """out = P psi, applying each single-wire Pauli matrix in turn."""
    out = copy(psi)
    for (w, letter) in paulis:
        apply_matrix(out, PAULI[letter], [w])
    return out


class CSRObservable:
    """A general sparse observable (the SparseHamiltonian of Sec. 2.2): row
    pointers, column indices and complex values of a 2^n x 2^n matrix.
    (H psi)_i = sum over the row's stored entries of value * psi[column]."""

    def __init__(self, indptr, indices, values):
        self.indptr = np.asarray(indptr, dtype=np.int64)
        self.indices = np.asarray(indices, dtype=np.int64)
        self.values = np.asarray(values, dtype=np.complex128)

    def apply(self, psi: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.indptr.size - 1), np.diff(self.indptr))
        out = np.zeros_like(psi)
        np.add.at(out, rows, self.values * psi[self.indices])
        return out


class MatrixObservable:
    """An observable given as a Hermitian 2^k x 2^k matrix on k wires (wires[0]
    = the matrix's most significant index bit), identity elsewhere: A psi is
    the plain dense application of the matrix to every group of amplitudes."""

    def __init__(self, wires, matrix):
        self.wires = [int(w) for w in wires]
        self.matrix = np.array(matrix, dtype=np.complex128)

    def apply(self, psi: np.ndarray) -> np.ndarray:
        return apply_matrix(copy(psi), self.matrix, self.wires)


def apply_hamiltonian(psi: np.ndarray, terms) -> np.ndarray:
    """out = sum_t c_t P_t psi (or H psi for a sparse observable)."""
    if hasattr(terms, "apply"):
        return terms.apply(psi)
    out = np.zeros_like(psi)
    for t in terms:
        axpy(out, apply_pauli_word(psi, t.paulis), t.coeff)
    return out


def expval(psi: np.ndarray, terms) -> float:
    """<psi|H|psi> = sum_t c_t <psi|P_t|psi> (each term's value is real); for a
    sparse observable the real part of <psi|H psi>."""
    if hasattr(terms, "apply"):
        return inner(psi, terms.apply(psi)).real
    e = 0.0
    for t in terms:
        e += t.coeff * inner(psi, apply_pauli_word(psi, t.paulis)).real
    return e


def variance(psi: np.ndarray, terms) -> float:
    """Var(H) = <psi|H^2|psi> - <psi|H|psi>^2, the variance measurement of the
    GPU device (Sec. 2.2), with H^2 psi formed as H applied twice."""
    h = apply_hamiltonian(psi, terms)
    h2 = apply_hamiltonian(h, terms)
    e = inner(psi, h).real
    return inner(psi, h2).real - e * e


def probabilities(psi: np.ndarray, wires: Sequence[int]) -> np.ndarray:
    """Marginal probabilities of measuring `wires` in the computational basis
    (the device's probability measurement, Sec. 2.2; Listing 3 reads them out):
    p[b] = sum over indices i whose bits at `wires` spell b of |psi_i|^2, with
    wires[0] the most significant bit of b and wire w at index bit n-1-w."""
    n = _nqubits(psi)
    k = len(wires)
    idx = np.arange(psi.size, dtype=np.int64)
    b = np.zeros(psi.size, dtype=np.int64)
    for j, w in enumerate(wires):
        b |= ((idx >> (n - 1 - w)) & 1) << (k - 1 - j)
    p = np.zeros(1 << k)
    np.add.at(p, b, psi.real ** 2 + psi.imag ** 2)
    return p


def sample(psi: np.ndarray, wires: Sequence[int], uniforms: Sequence[float]) -> np.ndarray:
    """Outcomes for given uniforms u in [0, 1): the first b whose cumulative
    probability (summed in ascending b) exceeds u * total (inverse transform)."""
    p = probabilities(psi, wires)
    cdf = np.cumsum(p)
    u = np.asarray(uniforms, dtype=np.float64) * cdf[-1]
    return np.minimum(np.searchsorted(cdf, u, side="right"), p.size - 1).astype(np.uint64)


def expvals(psi: np.ndarray, observables) -> np.ndarray:
    return np.array([expval(psi, H) for H in observables])


def norm2(psi: np.ndarray) -> float:
    return inner(psi, psi).real


# ---------------------------------------------------------------------------
# Adjoint Jacobian
# ---------------------------------------------------------------------------
class _Step:
    """One single-angle (or angle-free) operation of the expanded tape."""

    __slots__ = ("name", "wires", "controls", "cvals", "param", "scale", "adjoint", "matrix")

    def __init__(self, name, wires, controls, cvals, param, scale, adjoint, matrix=None):
        self.name, self.wires, self.controls, self.cvals = name, wires, controls, cvals
        self.param, self.scale, self.adjoint, self.matrix = param, scale, adjoint, matrix


def expand(ops) -> List[_Step]:
    """Rot -> RZ(phi), RY(theta), RZ(omega) (reversed, each inverted, under ``adjoint``)."""
    out: List[_Step] = []
    for op in ops:
        cv = op.ctrl_values
        if op.name == "Rot":
            parts = [("RZ", op.params[0]), ("RY", op.params[1]), ("RZ", op.params[2])]
            if op.adjoint:
                parts = parts[::-1]
            for g, p in parts:
                out.append(_Step(g, op.wires, op.controls, cv, p, op.scale, op.adjoint))
        elif op.name == "QubitUnitary":
            out.append(_Step(op.name, op.wires, op.controls, cv, None, 1.0, op.adjoint,
                             np.array(op.matrix, dtype=np.complex128)))
        else:
            p = op.params[0] if op.params else None
            out.append(_Step(op.name, op.wires, op.controls, cv, p, op.scale, op.adjoint))
    return out


def _step_matrix(st: _Step, params) -> np.ndarray:
    if st.matrix is not None:
        M = st.matrix
    else:
        ang = [] if st.param is None else [st.scale * float(params[st.param])]
        M = gate_matrix(st.name, ang)
    return M.conj().T.copy() if st.adjoint else M


def adjoint_jacobian(circuit, params: np.ndarray, observables=None, psi_final=None, clock=None):
    """(E, J): E[j] = <psi|O_j|psi>, J[j, p] = dE_j / dparams[p]  (adjoint method).

    ``clock``: an optional dict; wall seconds are added under "forward",
    "lambda" (lambda_j = O_j phi and E), "phi" (mu = G phi and phi's
    un-apply: the work done once) and "rows" (inner products and the lambdas'
    un-apply: the work done once per observable)."""
    obs = circuit.observables if observables is None else observables
    steps = expand(circuit.ops)
    t = {"forward": 0.0, "lambda": 0.0, "phi": 0.0, "rows": 0.0}
    t0 = time.perf_counter()
    phi = forward(circuit, params) if psi_final is None else copy(psi_final)
    t1 = time.perf_counter()
    t["forward"] += t1 - t0
    lams = [apply_hamiltonian(phi, H) for H in obs]
    E = np.array([inner(phi, lam).real for lam in lams])
    t0 = time.perf_counter()
    t["lambda"] += t0 - t1
    J = np.zeros((len(obs), circuit.n_params))
    for st in reversed(steps):
        M = _step_matrix(st, params)
        if st.param is not None:
            G, s = generator(st.name)
            if st.adjoint:
                s = -s
            mu = copy(phi)
            apply_matrix(mu, G, st.wires, st.controls, st.cvals)
            if st.controls:
                project_controls(mu, st.controls, st.cvals)
            t1 = time.perf_counter()
            t["phi"] += t1 - t0
            for j, lam in enumerate(lams):
                J[j, st.param] += st.scale * (-2.0 * s) * inner(lam, mu).imag
            del mu  # three vectors at a time (phi, lambda, mu), not four
            t0 = time.perf_counter()
            t["rows"] += t0 - t1
        Md = M.conj().T.copy()
        apply_matrix(phi, Md, st.wires, st.controls, st.cvals)
        t1 = time.perf_counter()
        t["phi"] += t1 - t0
        for lam in lams:
            apply_matrix(lam, Md, st.wires, st.controls, st.cvals)
        t0 = time.perf_counter()
        t["rows"] += t0 - t1
    if clock is not None:
        for k, v in t.items():
            clock[k] = clock.get(k, 0.0) + v
    return E, J


def jvp(circuit, params: np.ndarray, tangent: Sequence[float], observables=None) -> np.ndarray:
    """Forward-mode derivative along `tangent` (the Jacobian-vector product the
    paper names as future work in Sec. 5): psi and dpsi = d psi(params + t
    tangent)/dt at t = 0 go through the expanded tape together.  A step
    U = exp(i s theta G) with theta = scale * params[p] gives
    dpsi <- U dpsi + i s scale tangent[p] G (U psi); then
    d<H_j>/dt = 2 Re <psi|H_j|dpsi>."""
    obs = circuit.observables if observables is None else observables
    v = np.asarray(tangent, dtype=np.float64)
    psi = initial_state(circuit)
    dpsi = np.zeros_like(psi)
    for st in expand(circuit.ops):
        M = _step_matrix(st, params)
        apply_matrix(psi, M, st.wires, st.controls, st.cvals)
        apply_matrix(dpsi, M, st.wires, st.controls, st.cvals)
        if st.param is not None and v[st.param] != 0.0:
            G, s = generator(st.name)
            if st.adjoint:
                s = -s
            mu = copy(psi)
            apply_matrix(mu, G, st.wires, st.controls, st.cvals)
            if st.controls:
                project_controls(mu, st.controls, st.cvals)
            axpy(dpsi, mu, 1j * s * st.scale * v[st.param])
    return np.array([2.0 * inner(psi, apply_hamiltonian(dpsi, H)).real for H in obs])


def adjoint_vjp(circuit, params: np.ndarray, grad_out: Sequence[float], observables=None):
    """sum_j grad_out[j] * J[j, :] with one lambda = sum_j grad_out[j] O_j phi."""
    obs = circuit.observables if observables is None else observables
    merged = []
    for g, H in zip(grad_out, obs):
        for t in H:
            merged.append(type(t)(float(g) * t.coeff, t.paulis))
    _, J = adjoint_jacobian(circuit, params, [merged])
    return J[0]


# ---------------------------------------------------------------------------
# Shift / finite-difference gradients
# ---------------------------------------------------------------------------
TWO_TERM = {"RX", "RY", "RZ", "PhaseShift", "IsingXX", "IsingYY", "IsingZZ", "Rot"}


def _with_shifted_use(circuit, params, op_index, slot, shift):
    """Copy of (ops, params) where only one use of one angle is shifted."""
    import dataclasses
    ops = list(circuit.ops)
    op = ops[op_index]
    newp = np.concatenate([params, [params[op.params[slot]] + shift / op.scale]])
    idx = list(op.params)
    idx[slot] = len(params)
    ops[op_index] = dataclasses.replace(op, params=tuple(idx))
    c2 = dataclasses.replace(circuit, ops=ops, n_params=len(newp))
    return c2, newp


def param_shift_jacobian(circuit, params: np.ndarray, observables=None):
    """Two-term shift rule (shift pi/2, factor 1/2) per angle use; uncontrolled
    Pauli-rotation family only (generator eigenvalues with a single frequency)."""
    obs = circuit.observables if observables is None else observables
    J = np.zeros((len(obs), circuit.n_params))
    for k, op in enumerate(circuit.ops):
        if not op.params:
            continue
        if op.name not in TWO_TERM or op.controls:
            raise ValueError(f"two-term shift rule does not apply to {op.name} with controls={op.controls}")
        for slot in range(len(op.params)):
            cp, pp = _with_shifted_use(circuit, params, k, slot, math.pi / 2)
            cm, pm = _with_shifted_use(circuit, params, k, slot, -math.pi / 2)
            ep = expvals(forward(cp, pp), obs)
            em = expvals(forward(cm, pm), obs)
            J[:, op.params[slot]] += op.scale * 0.5 * (ep - em)
    return J


def finite_diff_jacobian(circuit, params: np.ndarray, observables=None, h: float = 1e-5):
    """Central differences in every parameter (sanity check only)."""
    obs = circuit.observables if observables is None else observables
    J = np.zeros((len(obs), circuit.n_params))
    for p in range(circuit.n_params):
        pp = params.copy()
        pp[p] += h
        pm = params.copy()
        pm[p] -= h
        J[:, p] = (expvals(forward(circuit, pp), obs) - expvals(forward(circuit, pm), obs)) / (2 * h)
    return J
