"""Seeded circuit / observable generators for the five workload shapes.

Conventions shared by every consumer (they are conventions of description,
not of arithmetic):

* a circuit acts on ``n`` wires; wire 0 is the most significant bit of an
  amplitude index (Alg. 1 sets q_offset = n - q - 1);
* an :class:`Op` names a base gate, its target wires, optional control wires
  and control values (Alg. 2 and its "prescribed bit string"), the indices of
  its angles in the circuit's parameter array, an angle scale
  (angle = scale * params[index]) and the ``inverse`` / adjoint flag of
  Listing 1;
* an observable is a list of :class:`Term` (coefficient, Pauli letters per
  wire), i.e. a Hamiltonian of coefficients and tensor-product Pauli words as
  in Listing 2;
* a :class:`MatrixOp` is a fixed dense 2^k x 2^k unitary on k wires (the
  QubitUnitary of the gate list), given as data; its matrix index has wires[0]
  as the most significant bit.

Gate names follow the paper's gate list (Section 2.1.2): PauliX, PauliY,
PauliZ, Hadamard, S, T, PhaseShift, RX, RY, RZ, Rot, SWAP, IsingXX, IsingXY,
IsingYY, IsingZZ, plus the Givens gates SingleExcitation / DoubleExcitation of
the VQE section.  Controlled gates (CNOT, CZ, CRX, ...) are a base gate with
control wires.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

# number of target wires per base gate
GATE_ARITY = {
    "Identity": 1, "PauliX": 1, "PauliY": 1, "PauliZ": 1, "Hadamard": 1,
    "S": 1, "T": 1, "PhaseShift": 1, "RX": 1, "RY": 1, "RZ": 1, "Rot": 1,
    "SWAP": 2, "IsingXX": 2, "IsingYY": 2, "IsingZZ": 2, "IsingXY": 2,
    "SingleExcitation": 2, "DoubleExcitation": 4,
}

# number of angles per base gate
GATE_NPARAMS = {
    "Identity": 0, "PauliX": 0, "PauliY": 0, "PauliZ": 0, "Hadamard": 0,
    "S": 0, "T": 0, "PhaseShift": 1, "RX": 1, "RY": 1, "RZ": 1, "Rot": 3,
    "SWAP": 0, "IsingXX": 1, "IsingYY": 1, "IsingZZ": 1, "IsingXY": 1,
    "SingleExcitation": 1, "DoubleExcitation": 1,
}

PARAMETRIC = [g for g, k in GATE_NPARAMS.items() if k > 0]
CONSTANT = [g for g, k in GATE_NPARAMS.items() if k == 0]


@dataclass(frozen=True)
class Op:
    name: str
    wires: Tuple[int, ...]
    params: Tuple[int, ...] = ()
    controls: Tuple[int, ...] = ()
    control_values: Tuple[int, ...] = ()
    adjoint: bool = False
    scale: float = 1.0

    def __post_init__(self):
        if self.name not in GATE_ARITY:
            raise ValueError(f"unknown gate {self.name}")
        if len(self.wires) != GATE_ARITY[self.name]:
            raise ValueError(f"{self.name} takes {GATE_ARITY[self.name]} wires")
        if len(self.params) != GATE_NPARAMS[self.name]:
            raise ValueError(f"{self.name} takes {GATE_NPARAMS[self.name]} params")
        if self.control_values and len(self.control_values) != len(self.controls):
            raise ValueError("control_values must match controls")

    @property
    def ctrl_values(self) -> Tuple[int, ...]:
        return self.control_values if self.control_values else (1,) * len(self.controls)


@dataclass(frozen=True)
class MatrixOp:
    """A fixed dense unitary on ``wires`` (no angles): ``matrix`` is 2^k x 2^k,
    row / column bit j (from the most significant) belongs to wires[j]."""
    wires: Tuple[int, ...]
    matrix: np.ndarray = field(compare=False, repr=False)
    controls: Tuple[int, ...] = ()
    control_values: Tuple[int, ...] = ()
    adjoint: bool = False
    name: str = "QubitUnitary"
    params: Tuple[int, ...] = ()
    scale: float = 1.0

    def __post_init__(self):
        if self.name != "QubitUnitary":
            raise ValueError("MatrixOp is a QubitUnitary")
        if np.shape(self.matrix) != (1 << len(self.wires), 1 << len(self.wires)):
            raise ValueError("matrix must be 2^k x 2^k for k wires")
        if self.control_values and len(self.control_values) != len(self.controls):
            raise ValueError("control_values must match controls")

    @property
    def ctrl_values(self) -> Tuple[int, ...]:
        return self.control_values if self.control_values else (1,) * len(self.controls)


def random_unitary(k: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed 2^k x 2^k unitary (input data): QR of a complex Gaussian
    matrix with the phases of R's diagonal moved into Q (Mezzadri, Notices AMS
    54, 2007)."""
    d = 1 << k
    z = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)


@dataclass(frozen=True)
class Term:
    coeff: float
    paulis: Tuple[Tuple[int, str], ...]  # ((wire, 'X'|'Y'|'Z'), ...), wires distinct


@dataclass
class Circuit:
    n: int
    ops: List[Op]
    n_params: int
    observables: List[List[Term]] = field(default_factory=list)
    basis_state: int = 0          # initial |basis_state>, index with wire 0 = MSB
    name: str = ""

    def n_gates(self) -> int:
        return len(self.ops)


def config_seed(index: int) -> int:
    """Seed of workload shape ``index`` (1-based, in the order they are listed)."""
    return 240302512 + index


def _z(w: int) -> List[Term]:
    return [Term(1.0, ((w, "Z"),))]


# ---------------------------------------------------------------------------
# Layered RX/RY/RZ + CNOT ladder
# ---------------------------------------------------------------------------
def layered_circuit(n: int = 12, layers: int = 10, seed: int | None = None):
    """RX, RY, RZ on every wire then CNOT(i, i+1) per layer; O = sum_i Z_i.

    Returns (circuit, params) with angles uniform in [0, 2pi).
    """
    rng = np.random.default_rng(config_seed(1) if seed is None else seed)
    ops: List[Op] = []
    p = 0
    for _ in range(layers):
        for w in range(n):
            for g in ("RX", "RY", "RZ"):
                ops.append(Op(g, (w,), (p,)))
                p += 1
        for i in range(n - 1):
            ops.append(Op("PauliX", (i + 1,), controls=(i,)))
    params = rng.uniform(0.0, 2.0 * np.pi, size=p)
    obs = [[Term(1.0, ((w, "Z"),)) for w in range(n)]]
    return Circuit(n, ops, p, obs, name=f"layered_n{n}_l{layers}"), params


# ---------------------------------------------------------------------------
# Strongly-entangling layers
# ---------------------------------------------------------------------------
def strongly_entangling(n: int = 24, layers: int = 8, seed: int | None = None):
    """Rot(phi, theta, omega) per wire then CNOT(i, (i+r) mod n), r = l mod (n-1) + 1.

    Observables: the n single-wire Z_j.  Angles uniform in [0, 2pi).
    """
    rng = np.random.default_rng(config_seed(2) if seed is None else seed)
    ops: List[Op] = []
    p = 0
    for l in range(layers):
        for w in range(n):
            ops.append(Op("Rot", (w,), (p, p + 1, p + 2)))
            p += 3
        r = (l % (n - 1)) + 1
        for i in range(n):
            ops.append(Op("PauliX", ((i + r) % n,), controls=(i,)))
    params = rng.uniform(0.0, 2.0 * np.pi, size=p)
    obs = [_z(w) for w in range(n)]
    return Circuit(n, ops, p, obs, name=f"sel_n{n}_l{layers}"), params


# ---------------------------------------------------------------------------
# QAOA MaxCut
# ---------------------------------------------------------------------------
def regular_graph(n: int, rng: np.random.Generator, degree: int = 3):
    """Seeded simple graph with every vertex of degree 3.

    For odd n (no 3-regular graph exists) one vertex gets degree 2, giving
    (3n - 1) / 2 edges.  Pairing model with rejection of loops / multi-edges.
    """
    deg = [degree] * n
    if (degree * n) % 2 == 1:
        deg[-1] = degree - 1
    for _ in range(10000):
        stubs = np.repeat(np.arange(n), deg)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)
    raise RuntimeError("could not draw a simple regular graph")


def qaoa_maxcut(n: int = 20, p: int = 4, seed: int | None = None, edges=None):
    """QAOA MaxCut circuit: H on all wires, then p x (IsingZZ(2 gamma_l) per edge, RX(2 beta_l) per wire).

    Parameter layout: params[0:p] = gamma, params[p:2p] = beta.
    Observable H_C = sum over edges of Z_u Z_v.
    """
    rng = np.random.default_rng(config_seed(3) if seed is None else seed)
    if edges is None:
        edges = regular_graph(n, rng)
    ops: List[Op] = [Op("Hadamard", (w,)) for w in range(n)]
    for l in range(p):
        for (u, v) in edges:
            ops.append(Op("IsingZZ", (u, v), (l,), scale=2.0))
        for w in range(n):
            ops.append(Op("RX", (w,), (p + l,), scale=2.0))
    obs = [[Term(1.0, ((u, "Z"), (v, "Z"))) for (u, v) in edges]]
    c = Circuit(n, ops, 2 * p, obs, name=f"qaoa_n{n}_p{p}")
    c.edges = list(edges)  # type: ignore[attr-defined]
    return c


def qaoa_param_sets(batch: int = 512, p: int = 4, seed: int | None = None):
    """``batch`` parameter sets (gamma, beta) uniform in [0, pi]^(2p)."""
    rng = np.random.default_rng((config_seed(3) if seed is None else seed) + 7)
    return rng.uniform(0.0, np.pi, size=(batch, 2 * p))


def qaoa_mixed_instances(count: int = 256, nmin: int = 14, nmax: int = 22, p: int = 4,
                         seed: int | None = None):
    """``count`` QAOA instances with n ~ U{nmin..nmax}, each with its own graph and angles."""
    rng = np.random.default_rng((config_seed(3) if seed is None else seed) + 11)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        edges = regular_graph(n, rng)
        c = qaoa_maxcut(n, p, seed=int(rng.integers(1 << 31)), edges=edges)
        params = rng.uniform(0.0, np.pi, size=2 * p)
        out.append((c, params))
    return out


# ---------------------------------------------------------------------------
# VQE-shaped Givens ansatz
# ---------------------------------------------------------------------------
def random_hamiltonian(n: int, n_terms: int, rng: np.random.Generator,
                       weights=(2, 3, 4), letters="XYZ") -> List[Term]:
    """Random Pauli sum: weight U{weights}, distinct wires, letters U{letters}, coeffs N(0,1)."""
    terms = []
    for _ in range(n_terms):
        w = int(rng.choice(weights))
        wires = rng.choice(n, size=min(w, n), replace=False)
        ls = rng.choice(list(letters), size=len(wires))
        paulis = tuple(sorted((int(a), str(b)) for a, b in zip(wires, ls)))
        terms.append(Term(float(rng.normal()), paulis))
    return terms


def vqe_givens(n: int = 24, electrons: int = 12, n_singles: int = 40, n_doubles: int = 120,
               n_terms: int = 2000, seed: int | None = None):
    """Hartree-Fock basis state plus DoubleExcitation / SingleExcitation gates.

    Occupied wires 0..electrons-1, virtual wires electrons..n-1.  Excitations
    conserve spin (even wires = one spin, odd wires = the other); doubles are
    applied before singles.  Angles N(0, 0.1).  Observable: a random
    ``n_terms`` Pauli sum.
    """
    rng = np.random.default_rng(config_seed(4) if seed is None else seed)
    occ = list(range(electrons))
    vir = list(range(electrons, n))
    singles = [(o, v) for o in occ for v in vir if o % 2 == v % 2]
    doubles = []
    for i, o1 in enumerate(occ):
        for o2 in occ[i + 1:]:
            for j, v1 in enumerate(vir):
                for v2 in vir[j + 1:]:
                    if (o1 % 2) + (o2 % 2) == (v1 % 2) + (v2 % 2):
                        doubles.append((o1, o2, v1, v2))
    n_singles = min(n_singles, len(singles))
    n_doubles = min(n_doubles, len(doubles))
    s_idx = rng.choice(len(singles), size=n_singles, replace=False)
    d_idx = rng.choice(len(doubles), size=n_doubles, replace=False)
    ops: List[Op] = []
    p = 0
    for k in d_idx:
        ops.append(Op("DoubleExcitation", doubles[int(k)], (p,)))
        p += 1
    for k in s_idx:
        ops.append(Op("SingleExcitation", singles[int(k)], (p,)))
        p += 1
    params = rng.normal(0.0, 0.1, size=p)
    ham = random_hamiltonian(n, n_terms, rng)
    hf = ((1 << electrons) - 1) << (n - electrons)  # wires 0..electrons-1 set (wire 0 = MSB)
    c = Circuit(n, ops, p, [ham], basis_state=hf, name=f"vqe_n{n}_e{electrons}")
    return c, params


# ---------------------------------------------------------------------------
# RY layers + CZ brick
# ---------------------------------------------------------------------------
def dense_block_wires(n: int, b: int) -> Tuple[int, ...]:
    """Wires of the b-th 5-qubit dense block of :func:`ry_cz_brick` (n >= 10):
    the top five wires, the bottom five (global index bit 0 among them), five
    scattered wires in descending order, then the middle five; repeating."""
    return [tuple(range(5)), tuple(range(n - 5, n)), (n - 2, 2 * n // 3, n // 2, n // 3, 1),
            tuple(range(n // 2 - 2, n // 2 + 3))][b % 4]


def ry_cz_brick(n: int = 30, layers: int = 20, seed: int | None = None, dense_every: int = 5):
    """RY on every wire then a CZ brick (even layer: CZ(2i, 2i+1); odd: CZ(2i+1, 2i+2)).

    After every ``dense_every``-th layer (0: none) comes a fixed 5-qubit dense
    block: a Haar-random unitary (a stand-in for a block fused from several
    gates) on the wires of :func:`dense_block_wires`.  Observable
    Z_0 Z_{n-1}.  Angles uniform in [0, 2pi); the blocks draw from a separate
    stream, so the angles do not depend on them.
    """
    seed = config_seed(5) if seed is None else seed
    rng = np.random.default_rng(seed)
    mrng = np.random.default_rng([seed, 5])
    ops: List = []
    p = 0
    blocks = 0
    for l in range(layers):
        for w in range(n):
            ops.append(Op("RY", (w,), (p,)))
            p += 1
        start = 0 if l % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            ops.append(Op("PauliZ", (a + 1,), controls=(a,)))
        if dense_every > 0 and (l + 1) % dense_every == 0:
            if n < 10:
                raise ValueError("dense blocks need n >= 10 (or dense_every=0)")
            ops.append(MatrixOp(dense_block_wires(n, blocks), random_unitary(5, mrng)))
            blocks += 1
    params = rng.uniform(0.0, 2.0 * np.pi, size=p)
    obs = [[Term(1.0, ((0, "Z"), (n - 1, "Z")))]]
    return Circuit(n, ops, p, obs, name=f"rycz_n{n}_l{layers}"), params


# ---------------------------------------------------------------------------
# Random circuits / states for tests
# ---------------------------------------------------------------------------
def random_circuit(n: int, n_ops: int, seed: int, gates: Sequence[str] | None = None,
                   max_controls: int = 2, p_control: float = 0.25, p_adjoint: float = 0.2,
                   shared_params: bool = False):
    """Random circuit over ``gates`` (default: every base gate that fits in n wires)."""
    rng = np.random.default_rng(seed)
    if gates is None:
        gates = [g for g in GATE_ARITY if GATE_ARITY[g] <= n and g != "Identity"]
    ops: List[Op] = []
    p = 0
    for _ in range(n_ops):
        g = str(rng.choice(list(gates)))
        k = GATE_ARITY[g]
        perm = [int(x) for x in rng.permutation(n)]
        wires = tuple(perm[:k])
        free = perm[k:]
        nc = 0
        if free and max_controls > 0 and rng.random() < p_control:
            nc = int(rng.integers(1, min(max_controls, len(free)) + 1))
        controls = tuple(free[:nc])
        cvals = tuple(int(v) for v in rng.integers(0, 2, size=nc)) if nc else ()
        npar = GATE_NPARAMS[g]
        if shared_params and p > 0 and rng.random() < 0.3:
            idx = tuple(int(rng.integers(0, p)) for _ in range(npar))
        else:
            idx = tuple(range(p, p + npar))
            p += npar
        scale = float(rng.choice([1.0, 1.0, 2.0, -0.5])) if npar else 1.0
        ops.append(Op(g, wires, idx, controls, cvals, bool(rng.random() < p_adjoint), scale))
    params = rng.uniform(-np.pi, np.pi, size=max(p, 0))
    return Circuit(n, ops, p, name=f"random_n{n}_s{seed}"), params


def random_state(n: int, seed: int) -> np.ndarray:
    """Seeded normalised random complex state (standard normal entries, then scaled)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)
