"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (tests/bars.py): complex128 expectation values 1e-10 and gradients
1e-9, each entry relative to max(|x|, 1e-3 max|x|); complex64 1e-4
normwise; amplitudes 1e-12 (complex128) and 1e-4 (complex64) absolute;
variances relative to <H^2>.
Sizes span several tiles (n > 11 local bits for complex128, > 12 for
complex64) and ragged cases (n = 1, 2, 3; empty tapes; zero-term observables).
"""

import math

import numpy as np
import pytest

import bars
import oracle
from oracle import dense
from workloads import (Circuit, Op, Term, GATE_ARITY, GATE_NPARAMS, layered_circuit, qaoa_maxcut,
                       random_circuit, random_hamiltonian, random_state, ry_cz_brick,
                       strongly_entangling, vqe_givens)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - GPU-only module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2403_02512_gb300 as svlib  # noqa: E402
from paper_2403_02512_gb300 import _lib as L  # noqa: E402
from paper_2403_02512_gb300.torch_api import Program, StateVector, expval as ad_expval  # noqa: E402

# "c128df": complex128 storage, double-float arithmetic -- held to the complex128 bars
DTYPES = ["c128", "c64", "c128df"]
TOL_STATE, TOL_E, TOL_J = bars.TOL_STATE, bars.TOL_E, bars.TOL_J


def _state(n, dtype, seed):
    sv = StateVector(n, dtype)
    psi = random_state(n, seed)
    sv.set_numpy(psi)
    # the oracle starts from exactly the amplitudes the GPU holds
    return sv, sv.to_numpy().astype(np.complex128)


def _assert_state(got, want, dtype):
    bars.check_state(got, want, dtype)


def _assert_rel(got, want, tol, what, dtype, magnitude=None):
    """The bar of `dtype` (entry-wise relative with a 1e-3 floor for complex128,
    normwise for complex64) at tolerance `tol`."""
    r = bars.check(got, want, dtype, tol, what, magnitude)
    bars.record(what, dtype, got, want, r)
    return r


# ---------------------------------------------------------------------------
# gates: every gate, every wire, controls, adjoint flag
# ---------------------------------------------------------------------------
GATES = [g for g in GATE_ARITY if g != "Identity"]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 13])
def test_single_gates_every_wire(dtype, n):
    rng = np.random.default_rng(1000 + n)
    for name in GATES:
        k = GATE_ARITY[name]
        if k > n:
            continue
        trials = n if n <= 5 else 6
        for trial in range(trials):
            wires = tuple(int(w) for w in rng.permutation(n)[:k]) if n > 5 else \
                tuple(int((trial + j) % n) for j in range(k))
            free = [w for w in range(n) if w not in wires]
            nc = min(len(free), trial % 3)
            controls = tuple(free[:nc])
            cvals = tuple(int(v) for v in rng.integers(0, 2, size=nc))
            npar = GATE_NPARAMS[name]
            op = Op(name, wires, tuple(range(npar)), controls, cvals, bool(trial % 2))
            params = rng.uniform(-4, 4, size=npar)
            sv, psi = _state(n, dtype, 7 * n + trial)
            L.sv_apply_op(sv.handle, L.Tape([op], npar).ops[0], params if npar else None)
            want = oracle.apply_op(psi.copy(), op, params)
            _assert_state(sv.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_sv_apply_plain_gates_and_matrices(dtype):
    n = 6
    sv, psi = _state(n, dtype, 3)
    sv.apply("RX", [2], [0.7]).apply("IsingXX", [0, 5], [1.3]).apply("Hadamard", [4]).apply("RZ", [1], [2.1], True)
    for op in (Op("RX", (2,), (0,)), Op("IsingXX", (0, 5), (0,)), Op("Hadamard", (4,)), Op("RZ", (1,), (0,), adjoint=True)):
        ang = {"RX": [0.7], "IsingXX": [1.3], "RZ": [2.1]}.get(op.name, [])
        oracle.apply_op(psi, op, np.array(ang))
    _assert_state(sv.to_numpy(), psi, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k", [1, 3, 5, 6])
def test_dense_matrix_blocks(dtype, k):
    n = 13
    rng = np.random.default_rng(k)
    A = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    U, _ = np.linalg.qr(A)
    wires = [int(w) for w in rng.permutation(n)[:k]]
    for adjoint in (False, True):
        sv, psi = _state(n, dtype, 40 + k)
        sv.apply_matrix(wires, U, adjoint)
        oracle.apply_matrix(psi, U.conj().T if adjoint else U, wires)
        _assert_state(sv.to_numpy(), psi, dtype)


# ---------------------------------------------------------------------------
# fused forward passes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,seed", [(3, 1), (7, 2), (12, 3), (14, 4)])
def test_random_circuit_forward(dtype, n, seed):
    c, p = random_circuit(n, 80, seed, max_controls=2)
    sv, psi = _state(n, dtype, seed)
    prog = Program(sv, c.ops, c.n_params)
    prog.forward(p, reset=False)
    _assert_state(sv.to_numpy(), oracle.forward(c, p, psi), dtype)


def test_empty_tape_leaves_the_state():
    sv, psi = _state(5, "c128", 9)
    L.sv_forward(sv.handle, L.Tape([], 0), np.zeros(0))
    assert np.array_equal(sv.to_numpy(), psi)


# ---------------------------------------------------------------------------
# expectation values
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 8, 9, 10, 13, 15])
def test_pauli_sum_expvals(dtype, n):
    # 43 words over 4 observables: complex128 sums them by observable (1, 2, 4 or 8
    # amplitudes per thread at these sizes), complex64 by word
    rng = np.random.default_rng(n)
    obs = [random_hamiltonian(n, 40, rng, weights=tuple(range(1, min(n, 4) + 1))),
           [Term(0.5, ())],                                 # identity term
           [],                                               # zero terms
           [Term(1.0, ((n - 1, "Y"),)), Term(-2.0, ((0, "X"),))]]
    sv, psi = _state(n, dtype, 100 + n)
    got = sv.expval(obs)
    want = np.array([oracle.expval(psi, H) for H in obs])
    _assert_rel(got, want, TOL_E[dtype], "expval", dtype)
    assert abs(sv.norm2() - oracle.norm2(psi)) <= TOL_E[dtype]


def test_expvals_repeat_bitwise():
    n = 16
    rng = np.random.default_rng(5)
    obs = [random_hamiltonian(n, 300, rng)]
    sv, _ = _state(n, "c128", 5)
    a, b = sv.expval(obs), sv.expval(obs)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# adjoint Jacobian, VJP, autograd
# ---------------------------------------------------------------------------
def _obs_for(n, rng):
    return [random_hamiltonian(n, 5, rng, weights=tuple(range(1, min(n, 3) + 1))),
            [Term(1.0, ((0, "Z"),))],
            random_hamiltonian(n, 3, rng, weights=(1,))]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,seed", [(2, 11), (4, 12), (7, 13), (12, 14), (13, 15)])
def test_adjoint_jacobian_random_circuits(dtype, n, seed):
    c, p = random_circuit(n, 40, seed, shared_params=True)
    rng = np.random.default_rng(seed)
    obs = _obs_for(n, rng)
    sv = StateVector(n, dtype)
    prog = Program(sv, c.ops, c.n_params, obs)
    prog.forward(p)
    E, J = prog.jacobian()
    Eo, Jo = oracle.adjoint_jacobian(c, p, obs)
    _assert_rel(E.cpu().numpy(), Eo, TOL_E[dtype], "expvals", dtype)
    _assert_rel(J.cpu().numpy(), Jo, TOL_J[dtype], "jacobian", dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_one_shot_jacobian_and_vjp_calls(dtype):
    n = 9
    c, p = random_circuit(n, 30, 21)
    rng = np.random.default_rng(21)
    obs = _obs_for(n, rng)
    h = L.sv_create(n, L.SV_C64 if dtype == "c64" else L.SV_C128)
    if dtype == "c128df":
        L.sv_set_compute(h, L.SV_COMPUTE_DOUBLE_FLOAT)
    try:
        tape, ps = L.Tape(c.ops, c.n_params), L.PauliSums(obs)
        L.sv_forward(h, tape, p)
        E, J = L.sv_adjoint_jacobian(h, tape, p, ps)
        g = rng.normal(size=len(obs))
        v = L.sv_adjoint_vjp(h, tape, p, ps, g)
    finally:
        L.sv_destroy(h)
    Eo, Jo = oracle.adjoint_jacobian(c, p, obs)
    _assert_rel(E, Eo, TOL_E[dtype], "expvals", dtype)
    _assert_rel(J, Jo, TOL_J[dtype], "jacobian", dtype)
    _assert_rel(v, g @ Jo, TOL_J[dtype], "vjp", dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_lambda_chunking_matches_single_sweep(dtype, monkeypatch):
    n = 12
    c, p = strongly_entangling(n, 2, seed=3)
    sv = StateVector(n, dtype)
    full = Program.from_circuit(sv, c)
    full.forward(p)
    E1, J1 = full.jacobian()
    monkeypatch.setenv("SV_LAMBDA_CHUNK", "5")
    chunked = Program.from_circuit(sv, c)
    chunked.set_params(p)
    E2, J2 = chunked.jacobian()
    assert torch.equal(E1, E2)
    _assert_rel(J2.cpu().numpy(), J1.cpu().numpy(), 1e-6 if dtype == "c64" else 1e-12, "chunked", dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_autograd_function_backward_is_adjoint_vjp(dtype):
    n = 10
    c, p = strongly_entangling(n, 2, seed=8)
    sv = StateVector(n, dtype)
    prog = Program.from_circuit(sv, c)
    params = torch.tensor(p, dtype=torch.float64, device="cuda", requires_grad=True)
    E = ad_expval(params, prog)
    w = torch.linspace(-1, 1, E.numel(), dtype=torch.float64, device="cuda")
    (E * w).sum().backward()
    _, Jo = oracle.adjoint_jacobian(c, p)
    _assert_rel(params.grad.cpu().numpy(), w.cpu().numpy() @ Jo, TOL_J[dtype], "autograd grad", dtype)


def test_jacobian_repeats_bitwise():
    n = 13
    c, p = random_circuit(n, 30, 31)
    obs = _obs_for(n, np.random.default_rng(31))
    sv = StateVector(n, "c128")
    prog = Program(sv, c.ops, c.n_params, obs)
    prog.forward(p)
    E1, J1 = prog.jacobian()
    E2, J2 = prog.jacobian()
    assert torch.equal(E1, E2) and torch.equal(J1, J2)


# ---------------------------------------------------------------------------
# The five workload shapes at oracle-friendly sizes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DTYPES)
def test_layered_12_qubit_full_size(dtype):
    c, p = layered_circuit(12, 10)
    sv = StateVector(12, dtype)
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    E, J = prog.jacobian()
    Eo, Jo = oracle.adjoint_jacobian(c, p)
    _assert_rel(E.cpu().numpy(), Eo, TOL_E[dtype], "expvals", dtype)
    _assert_rel(J.cpu().numpy(), Jo, TOL_J[dtype], "jacobian", dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("maker", ["sel", "qaoa", "vqe", "rycz"])
def test_workload_shapes_small(dtype, maker):
    if maker == "sel":
        c, p = strongly_entangling(13, 3, seed=1)
    elif maker == "qaoa":
        c = qaoa_maxcut(14, 2, seed=2)
        p = np.random.default_rng(2).uniform(0, math.pi, size=4)
    elif maker == "vqe":
        c, p = vqe_givens(12, 6, 10, 20, 150, seed=3)
    else:
        # a 5-qubit dense block after every second layer: all four block windows
        # (complex64: the tensor cores, forward and un-applied in the sweep)
        c, p = ry_cz_brick(14, 8, seed=4, dense_every=2)
    sv = StateVector(c.n, dtype, basis_state=c.basis_state)
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    if maker == "vqe":
        amps = sv.to_numpy()
        weights = np.array([bin(i).count("1") for i in range(1 << c.n)])
        assert np.all(amps[weights != 6] == 0)          # Givens gates keep Hamming weight exactly
    E, J = prog.jacobian()
    Eo, Jo = oracle.adjoint_jacobian(c, p)
    _assert_rel(E.cpu().numpy(), Eo, TOL_E[dtype], "expvals", dtype)
    _assert_rel(J.cpu().numpy(), Jo, TOL_J[dtype], "jacobian", dtype)


def test_compute_mode_switch_rebuilds_matrices():
    n = 11
    c, p = strongly_entangling(n, 2, seed=4)
    sv = StateVector(n, "c128")
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    E1, J1 = prog.jacobian()
    L.sv_set_compute(sv.handle, L.SV_COMPUTE_DOUBLE_FLOAT)
    prog.forward(p)
    E2, J2 = prog.jacobian()
    _assert_rel(E2.cpu().numpy(), E1.cpu().numpy(), 1e-10, "expvals", "c128")
    _assert_rel(J2.cpu().numpy(), J1.cpu().numpy(), 1e-9, "jacobian", "c128")
    with pytest.raises(L.SvError):
        L.sv_set_compute(StateVector(3, "c64").handle, L.SV_COMPUTE_DOUBLE_FLOAT)


def test_program_refuses_to_run_before_parameters_are_set():
    c, p = strongly_entangling(4, 1, seed=1)
    sv = StateVector(4, "c128")
    prog = Program.from_circuit(sv, c)
    with pytest.raises(L.SvError) as ei:
        prog.jacobian()
    assert ei.value.status == 6
    prog.set_params(p)
    prog.jacobian()


def test_error_status_for_bad_calls():
    sv = StateVector(4, "c128")
    with pytest.raises(L.SvError) as ei:
        sv.apply("RX", [7], [0.1])
    assert ei.value.status == 1
    with pytest.raises(L.SvError):
        sv.apply("RX", [1], [float("nan")])
    with pytest.raises(L.SvError):
        sv.expval([[Term(1.0, ((9, "Z"),))]])
    L.sv_set_alloc_cap(1 << 20)
    try:
        with pytest.raises(L.SvError) as ei:
            L.sv_create(20, L.SV_C128)
        assert ei.value.status == 2
    finally:
        L.sv_set_alloc_cap(0)


# ---- renormalisation after a forward pass (complex64 precision reading) ------
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_renormalize_divides_by_the_fp64_norm(dtype):
    n = 13
    sv = StateVector(n, dtype, renormalize=True)
    psi = 2.0 * random_state(n, 71)  # ||psi||^2 = 4
    sv.set_numpy(psi)
    start = sv.to_numpy().astype(np.complex128)
    prog = Program(sv, [Op("PauliX", (0,))], 0)
    prog.set_params([])
    prog.forward(reset=False)
    want = oracle.forward(Circuit(n, [Op("PauliX", (0,))], 0, []), np.zeros(0), psi0=start)
    want = want / np.linalg.norm(want)
    _assert_state(sv.to_numpy(), want, dtype)
    assert abs(sv.norm2() - 1.0) <= (1e-6 if dtype == "c64" else 1e-14)


def test_renormalize_keeps_a_deep_complex64_circuit_on_the_unit_sphere():
    n = 14
    c, params = random_circuit(n, 600, 72)
    want = oracle.forward(c, params)
    drift = {}
    for on in (False, True):
        sv = StateVector(n, "c64", renormalize=on)
        prog = Program(sv, c.ops, c.n_params)
        prog.forward(params)
        got = sv.to_numpy()
        _assert_state(got, want, "c64")
        drift[on] = abs(sv.norm2() - 1.0)
    assert drift[True] <= 1e-6
    assert drift[True] <= drift[False] + 1e-7


def test_renormalize_flag_is_checked():
    import ctypes
    sv = StateVector(3, "c64")
    assert L.load().sv_set_renormalize(ctypes.c_void_p(sv.handle), 2) == 1  # SV_ERR_ARG
    assert L.load().sv_set_renormalize(None, 1) == 1


# ---- phase runs: adjacent RZ / IsingZZ with one angle as one diagonal --------
def _phase_run_circuit(n, seed):
    rng = np.random.default_rng(seed)
    ops = [Op("Hadamard", (w,)) for w in range(n)]
    # 40 IsingZZ on random wire pairs sharing parameter 0 (local and tile bits mixed)
    for _ in range(40):
        a, b = rng.choice(n, 2, replace=False)
        ops.append(Op("IsingZZ", (int(a), int(b)), (0,), scale=2.0))
    ops += [Op("RX", (w,), (1,)) for w in range(n)]
    # RZ run on a constant-free shared parameter, with the adjoint flag
    ops += [Op("RZ", (w,), (2,), adjoint=True) for w in range(0, n, 2)]
    # a run broken by a parameter change, then a 64-member run
    ops += [Op("RZ", (1,), (3,)), Op("RZ", (2,), (4,))]
    for _ in range(70):
        a, b = rng.choice(n, 2, replace=False)
        ops.append(Op("IsingZZ", (int(a), int(b)), (3,)))
    ops += [Op("RY", (w,), (4,)) for w in range(n)]
    return Circuit(n, ops, 5, [[Term(1.0, ((0, "Z"), (n - 1, "Z")))]]), rng.uniform(0, 2 * np.pi, 5)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [5, 16])
def test_phase_runs_forward_and_jacobian(dtype, n):
    c, p = _phase_run_circuit(n, 80 + n)
    sv = StateVector(n, dtype)
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    want = oracle.forward(c, p)
    _assert_state(sv.to_numpy(), want, dtype)
    E, J = prog.jacobian()
    _assert_rel(E.cpu().numpy(), oracle.expvals(want, c.observables), TOL_E[dtype], "expval", dtype)
    _assert_rel(J.cpu().numpy(), oracle.adjoint_jacobian(c, p)[1], TOL_J[dtype], "jacobian", dtype)


def test_phase_runs_in_a_batch():
    circs, params = [], []
    for i, n in enumerate((5, 12, 16)):
        c, p = _phase_run_circuit(n, 90 + i)
        circs.append(c)
        params.append(p)
    b = L.Batch(circs, L.SV_C64)
    b.set_params(np.concatenate(params))
    got = b.run()
    b.close()
    for c, p, g in zip(circs, params, got):
        want = oracle.expvals(oracle.forward(c, p), c.observables)[0]
        assert abs(g - want) <= 1e-4, (c.n, g, want)


# ---- variances ---------------------------------------------------------------
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 13, 18])
def test_variance_matches_oracle(dtype, n):
    sv, psi = _state(n, dtype, 300 + n)
    rng = np.random.default_rng(300 + n)
    obs = [random_hamiltonian(n, 25, rng, weights=tuple(range(1, min(n, 4) + 1))) for _ in range(3)]
    obs.append([Term(1.0, ((0, "Z"),))])          # single word: 1 - <Z>^2
    obs.append([Term(0.5, ())])                   # identity: variance 0
    obs.append([])                                # no terms: 0
    got = sv.var(obs)
    want = np.array([oracle.variance(psi, H) for H in obs])
    # Var = <H^2> - <H>^2: the rounding of the difference scales with <H^2>
    h2 = want + np.array([oracle.expval(psi, H) for H in obs]) ** 2
    _assert_rel(got, want, TOL_E[dtype], "variance", dtype, magnitude=h2)
    again = sv.var(obs)
    assert np.array_equal(got, again)             # fixed-order reductions repeat bitwise


# ---- observables given as Hermitian matrices ------------------------------------
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,wires", [(6, (2,)), (9, (8, 0)), (11, (3, 10, 5)), (12, (11, 6, 0, 2)),
                                     (13, (12, 1, 7, 4, 0))])
def test_hermitian_observables_as_pauli_words(dtype, n, wires):
    # the matrix's Pauli words (host decomposition) through the Pauli-sum
    # kernels, against the oracle applying the matrix itself
    rng = np.random.default_rng(800 + n)
    k = len(wires)
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    A = (a + a.conj().T) / 2
    H = L.sv_hermitian_to_pauli(n, wires, A)
    want_obs = oracle.MatrixObservable(wires, A)
    c, p = random_circuit(n, 30, 800 + n)
    sv = StateVector(n, dtype)
    prog = Program(sv, c.ops, c.n_params, [H])
    prog.forward(p)
    E, J = prog.jacobian()
    Eo, Jo = oracle.adjoint_jacobian(c, p, [want_obs])
    _assert_rel(E.cpu().numpy(), Eo, TOL_E[dtype], "expval", dtype)
    _assert_rel(J.cpu().numpy(), Jo, TOL_J[dtype], "jacobian", dtype)
    psi = oracle.forward(c, p)
    var_o = oracle.variance(psi, want_obs)
    _assert_rel(sv.var([H]), [var_o], TOL_E[dtype], "variance", dtype,
                magnitude=[var_o + oracle.expval(psi, want_obs) ** 2])


# ---- probabilities and samples -----------------------------------------------
def _wire_sets(n, rng):
    sets = [[], [0], [n - 1], list(range(n)), list(range(n))[::-1]]
    for k in (2, 3, min(n, 6)):
        if k <= n:
            sets.append([int(w) for w in rng.permutation(n)[:k]])
    return sets


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 13, 20])
def test_probabilities_match_oracle(dtype, n):
    sv, psi = _state(n, dtype, 400 + n)
    rng = np.random.default_rng(400 + n)
    for wires in _wire_sets(n, rng):
        got = sv.probs(wires)
        want = oracle.probabilities(psi, wires)
        assert got.shape == want.shape
        assert np.abs(got - want).max() <= 1e-12, wires
        assert np.array_equal(got, sv.probs(wires))  # fixed-order sums repeat bitwise


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [3, 13, 20])
def test_samples_match_oracle_inverse_transform(dtype, n):
    sv, psi = _state(n, dtype, 500 + n)
    rng = np.random.default_rng(500 + n)
    for wires in _wire_sets(n, rng):
        u = rng.random(4000)
        got = sv.sample(wires, u)
        want = oracle.sample(psi, wires, u)
        # equal except where u * total lies within rounding of a CDF boundary
        # (the device's scan and the oracle's running sum round differently)
        cdf = np.cumsum(oracle.probabilities(psi, wires))
        target = u * cdf[-1]
        g = got.astype(np.int64)
        lo = np.where(g > 0, cdf[np.maximum(g - 1, 0)], 0.0)
        assert np.all(lo <= target + 1e-12) and np.all(cdf[g] > target - 1e-12), wires
        assert np.count_nonzero(got != want) <= 2, wires
        assert np.array_equal(got, sv.sample(wires, u))


def test_probabilities_and_samples_reject_bad_arguments():
    sv = StateVector(4, "c128")
    for wires in ([0, 0], [4], [-1]):
        with pytest.raises(L.SvError) as ei:
            sv.probs(wires)
        assert ei.value.status == 1
    for u in ([1.0], [-0.1], [float("nan")]):
        with pytest.raises(L.SvError) as ei:
            sv.sample([0], u)
        assert ei.value.status == 1
    assert sv.sample([0, 1], []).size == 0


# ---- forward-mode Jacobian-vector products -----------------------------------
def _jvp_cases():
    c1, p1 = random_circuit(7, 60, 61, max_controls=2, shared_params=True)
    c1 = Circuit(c1.n, c1.ops, c1.n_params, [random_hamiltonian(7, 10, np.random.default_rng(61), weights=(1, 2)),
                                              [Term(1.0, ((3, "Z"),))]])
    c2, p2 = random_circuit(13, 80, 62, max_controls=1)
    c2 = Circuit(c2.n, c2.ops, c2.n_params, [[Term(0.5, ((0, "X"), (12, "Y")))], [Term(1.0, ((6, "Z"),))]])
    c3, p3 = strongly_entangling(12, 2, seed=63)
    c4, p4 = qaoa_maxcut(12, 2), np.random.default_rng(64).uniform(0, np.pi, 4)
    return [(c1, p1), (c2, p2), (c3, p3), (c4, p4)]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", range(4))
def test_jvp_matches_oracle_forward_mode(dtype, case):
    c, p = _jvp_cases()[case]
    v = np.random.default_rng(70 + case).normal(size=c.n_params)
    sv = StateVector(c.n, dtype)
    prog = Program.from_circuit(sv, c)
    prog.set_params(p)
    got = prog.jvp(v).cpu().numpy()
    want = oracle.jvp(c, p, v)
    _assert_rel(got, want, TOL_J[dtype], "jvp", dtype)
    # the state ends as the forward output; the reverse-mode Jacobian agrees
    _assert_state(sv.to_numpy(), oracle.forward(c, p), dtype)
    _, J = prog.jacobian()
    _assert_rel(J.cpu().numpy() @ v, got, TOL_J[dtype], "J @ v", dtype)


def test_jacobian_by_shape_uses_forward_mode_when_parameters_are_few():
    n = 9
    ops = [Op("RY", (w,), (w % 3,)) for w in range(n)] + [Op("PauliX", (w + 1,), controls=(w,)) for w in range(n - 1)]
    obs = [[Term(1.0, ((w, "Z"),))] for w in range(n)]
    c = Circuit(n, ops, 3, obs)
    p = np.array([0.3, 1.2, 2.2])
    sv = StateVector(n, "c128")
    prog = Program.from_circuit(sv, c)
    prog.set_params(p)
    E, J = prog.jacobian_by_shape()  # 3 parameters < 9 observables: three tangent passes
    Eo, Jo = oracle.adjoint_jacobian(c, p)
    _assert_rel(E.cpu().numpy(), Eo, 1e-10, "expval", "c128")
    _assert_rel(J.cpu().numpy(), Jo, 1e-9, "jacobian", "c128")


def test_jvp_rejects_bad_tangents():
    c, p = strongly_entangling(4, 1, seed=65)
    sv = StateVector(4, "c128")
    prog = Program.from_circuit(sv, c)
    prog.set_params(p)
    bad = np.zeros(c.n_params)
    bad[2] = np.nan
    with pytest.raises(L.SvError) as ei:
        prog.jvp(bad)
    assert ei.value.status == 1


# ---- sparse (CSR) observables ----------------------------------------------------
def _random_sparse_hermitian(n, seed, entries=200):
    rng = np.random.default_rng(seed)
    N = 1 << n
    d = {}
    for _ in range(entries):
        i, j = (int(x) for x in rng.integers(0, N, 2))
        z = complex(rng.normal(), rng.normal()) if i != j else complex(rng.normal(), 0.0)
        d[(i, j)] = d.get((i, j), 0) + z
        if i != j:
            d[(j, i)] = d.get((j, i), 0) + z.conjugate()
    keys = sorted(d)
    rows = np.array([k[0] for k in keys], dtype=np.int64)
    cols = np.array([k[1] for k in keys], dtype=np.int64)
    vals = np.array([d[k] for k in keys], dtype=np.complex128)
    indptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    return np.cumsum(indptr), cols, vals


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [3, 13])
def test_sparse_expval_and_jacobian_match_oracle(dtype, n):
    indptr, cols, vals = _random_sparse_hermitian(n, 600 + n, entries=40 * n)
    H = oracle.CSRObservable(indptr, cols, vals)
    sp = L.Sparse(n, indptr, cols, vals)
    c, p = random_circuit(n, 40, 600 + n, max_controls=1)
    sv = StateVector(n, dtype)
    prog = Program(sv, c.ops, c.n_params)
    prog.forward(p)
    psi = oracle.forward(c, p)
    e = L.sv_sparse_expval(sv.handle, sp)
    want_e = oracle.expval(psi, H)
    _assert_rel([e], [want_e], TOL_E[dtype], "sparse expval", dtype)
    e2, J = L.sv_adjoint_jacobian_sparse(sv.handle, L.Tape(c.ops, c.n_params), p, sp)
    Eo, Jo = oracle.adjoint_jacobian(c, p, [H])
    _assert_rel([e2], Eo, TOL_E[dtype], "sparse expval (adjoint call)", dtype)
    _assert_rel(J, Jo[0], TOL_J[dtype], "sparse jacobian", dtype)
    assert e == L.sv_sparse_expval(sv.handle, sp)  # fixed order: bitwise repeat
    sp.close()


def test_sparse_observable_from_a_pauli_sum_agrees_with_the_pauli_path():
    n = 6
    rng = np.random.default_rng(610)
    Hp = random_hamiltonian(n, 12, rng, weights=(1, 2, 3))
    M = dense.hamiltonian(n, Hp)
    rows, cols = np.nonzero(M)
    indptr = np.zeros((1 << n) + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    sp = L.Sparse(n, np.cumsum(indptr), cols, M[rows, cols])
    sv, psi = _state(n, "c128", 610)
    assert abs(L.sv_sparse_expval(sv.handle, sp) - sv.expval([Hp])[0]) <= 1e-12
    sp.close()


def test_sparse_observable_validation():
    n = 3
    indptr, cols, vals = _random_sparse_hermitian(n, 620, entries=10)
    bad = cols.copy()
    bad[0] = 1 << n
    with pytest.raises(L.SvError):
        L.Sparse(n, indptr, bad, vals)
    bad_ptr = indptr.copy()
    bad_ptr[-1] += 1
    with pytest.raises(L.SvError):
        L.Sparse(n, bad_ptr, cols, vals)
    sp = L.Sparse(n, indptr, cols, vals)
    sv = StateVector(n + 1, "c128")
    with pytest.raises(L.SvError):
        L.sv_sparse_expval(sv.handle, sp)
    sp.close()


# ---- dense 5-qubit blocks on the tensor cores (complex64) ----------------------
def _unitary(k, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    U, _ = np.linalg.qr(A)
    return U


@pytest.mark.parametrize("n,wires", [(5, [0, 1, 2, 3, 4]), (6, [5, 1, 3, 0, 2]), (12, [7, 8, 9, 10, 11]),
                                     (16, [15, 0, 9, 3, 12]), (17, [2, 11, 5, 16, 8]),
                                     (14, [0, 3, 6, 9, 12])])  # last: no target on index bit 0
def test_dense5_tensor_cores_match_oracle_and_cuda_cores(n, wires):
    U = _unitary(5, 700 + n)
    for adjoint in (False, True):
        got = {}
        for tc in (True, False):
            L.sv_set_dense_tensor_cores(tc)
            try:
                sv, psi = _state(n, "c64", 700 + n)
                sv.apply_matrix(wires, U, adjoint)
                got[tc] = sv.to_numpy()
                sv.close()
            finally:
                L.sv_set_dense_tensor_cores(True)
        oracle.apply_matrix(psi, U.conj().T if adjoint else U, wires)
        assert np.abs(got[True] - psi).max() <= 1e-5      # three TF32 products: FP32-level accuracy
        assert np.abs(got[True] - got[False]).max() <= 1e-5


class _MatrixOp:
    """A dense user matrix on the tape (the binding's QubitUnitary)."""

    def __init__(self, wires, matrix, controls=(), control_values=()):
        self.name, self.wires, self.matrix = "QubitUnitary", tuple(wires), matrix
        self.params, self.constants = (), ()
        self.controls, self.control_values = tuple(controls), tuple(control_values)
        self.adjoint, self.scale = False, 1.0


def test_dense5_tensor_cores_with_controls_and_in_a_jacobian():
    n = 13
    U = _unitary(5, 720)
    blk_wires, ctrl = (3, 9, 4, 11, 6), (0,)
    pre = [Op("RY", (w,), (w,)) for w in range(n)]
    post = [Op("RX", (w,), (n + w,)) for w in range(n)]
    P = 2 * n  # one parameter per gate: the two-term shift rule is exact
    obs = [[Term(1.0, ((3, "Z"),))], [Term(0.5, ((9, "X"), (4, "Y")))]]
    p = np.random.default_rng(720).uniform(0, 2 * np.pi, P)

    def oracle_energy(q):
        psi = oracle.forward(Circuit(n, pre, P, []), q)
        oracle.apply_matrix(psi, U, list(blk_wires), list(ctrl), [1])
        psi = oracle.forward(Circuit(n, post, P, []), q, psi0=psi)
        return oracle.expvals(psi, obs), psi

    Eo, want = oracle_energy(p)
    Jo = np.zeros((2, P))
    for q in range(P):
        e = np.zeros(P)
        e[q] = 0.5 * np.pi
        Jo[:, q] = 0.5 * (oracle_energy(p + e)[0] - oracle_energy(p - e)[0])
    sv = StateVector(n, "c64")
    prog = Program(sv, pre + [_MatrixOp(blk_wires, U, ctrl, (1,))] + post, P, obs)
    prog.forward(p)
    _assert_state(sv.to_numpy(), want, "c64")
    E, J = prog.jacobian()  # the sweep un-applies the block with its adjoint on the tensor cores
    _assert_rel(E.cpu().numpy(), Eo, 1e-4, "expval", "c64")
    _assert_rel(J.cpu().numpy(), Jo, 1e-4, "jacobian", "c64")


@pytest.mark.parametrize("dtype", DTYPES)
def test_wide_dense_blocks_in_a_jacobian(dtype):
    # 6-qubit user matrix: a wide dense step outside the tiles, un-applied in the sweep
    n = 12
    U = _unitary(6, 730)
    blk_wires = (1, 10, 4, 7, 2, 11)
    pre = [Op("RY", (w,), (w,)) for w in range(n)]
    post = [Op("RZ", (w,), (n + w,)) for w in range(n)] + [Op("RX", (w,), (2 * n + w,)) for w in range(n)]
    P = 3 * n  # one parameter per gate: the two-term shift rule is exact
    obs = [[Term(1.0, ((10, "Z"),))]]
    p = np.random.default_rng(730).uniform(0, 2 * np.pi, P)

    def oracle_energy(q):
        psi = oracle.forward(Circuit(n, pre, P, []), q)
        oracle.apply_matrix(psi, U, list(blk_wires))
        psi = oracle.forward(Circuit(n, post, P, []), q, psi0=psi)
        return oracle.expvals(psi, obs)

    Eo = oracle_energy(p)
    Jo = np.zeros((1, P))
    for q in range(P):
        e = np.zeros(P)
        e[q] = 0.5 * np.pi
        Jo[:, q] = 0.5 * (oracle_energy(p + e) - oracle_energy(p - e))
    sv = StateVector(n, dtype)
    prog = Program(sv, pre + [_MatrixOp(blk_wires, U)] + post, P, obs)
    prog.forward(p)
    E, J = prog.jacobian()
    _assert_rel(E.cpu().numpy(), Eo, TOL_E[dtype], "expval", dtype)
    _assert_rel(J.cpu().numpy(), Jo, TOL_J[dtype], "jacobian", dtype)


# ---- Z-only words: one Walsh-Hadamard transform of |psi|^2 per thread and tile ----------
def _z_words(n, rng, count, max_weight=4):
    terms = []
    for _ in range(count):
        k = int(rng.integers(1, min(n, max_weight) + 1))
        wires = sorted(int(w) for w in rng.choice(n, size=k, replace=False))
        terms.append(Term(float(rng.normal()), tuple((w, "Z") for w in wires)))
    return terms


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [7, 8, 9, 12, 13, 17, 20])
def test_z_only_observables(dtype, n):
    # tile sizes T = min(n, 11 or 12) cover every transform width 2^(T - 8) (and the
    # general kernel below T = 8); 40 words exceed one chunk of 32, 600 exceed one pass
    rng = np.random.default_rng(900 + n)
    obs = [[Term(1.0, ((w, "Z"),))] for w in (0, n // 2, n - 1)]        # single Z on high, middle, low bits
    obs.append(_z_words(n, rng, 40))
    obs.append(_z_words(n, rng, 600))
    obs.append(_z_words(n, rng, 12) + random_hamiltonian(n, 12, rng, weights=tuple(range(1, min(n, 3) + 1))))
    obs.append([Term(0.7, ())] + _z_words(n, rng, 5))                   # identity word among Z words
    sv, psi = _state(n, dtype, 900 + n)
    got = sv.expval(obs)
    want = np.array([oracle.expval(psi, H) for H in obs])
    _assert_rel(got, want, TOL_E[dtype], "z-only expval", dtype)
    assert np.array_equal(got, sv.expval(obs))  # fixed-order sums repeat bitwise


# ---- single-wire trainable layers of every kind, adjoint flags, CNOT layers --------------
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n_obs", [1, 3])
def test_single_wire_layers_jacobian(dtype, n_obs):
    # one and three observables: one lambda per CTA (the VJP shape) and several
    n = 13
    rng = np.random.default_rng(950 + n_obs)
    names = ["RX", "RY", "RZ", "PhaseShift", "Rot", "Hadamard"]
    ops, p = [], 0
    for layer in range(4):
        for w in rng.permutation(n):
            g = names[int(rng.integers(0, len(names)))]
            npar = GATE_NPARAMS[g]
            ops.append(Op(g, (int(w),), tuple(range(p, p + npar)), adjoint=bool(rng.integers(0, 2))))
            p += npar
        ops += [Op("PauliX", ((w + 1 + layer) % n,), controls=(w,)) for w in range(0, n, 3)]
    obs = [[Term(1.0, ((int(rng.integers(0, n)), "Z"),))] for _ in range(n_obs - 1)]
    obs.insert(0, random_hamiltonian(n, 6, rng, weights=(1, 2)))
    c = Circuit(n, ops, p, obs)
    params = rng.uniform(0, 2 * np.pi, p)
    sv = StateVector(n, dtype)
    prog = Program.from_circuit(sv, c)
    prog.forward(params)
    E, J = prog.jacobian()
    Eo, Jo = oracle.adjoint_jacobian(c, params)
    _assert_rel(E.cpu().numpy(), Eo, TOL_E[dtype], "expvals", dtype)
    _assert_rel(J.cpu().numpy(), Jo, TOL_J[dtype], "jacobian", dtype)
    g = rng.normal(size=n_obs)
    _assert_rel(prog.vjp(g).cpu().numpy(), g @ Jo, TOL_J[dtype], "vjp", dtype)


def test_closing_a_state_first_closes_its_programs():
    # a program refers to its state: closing the state closes the program with it
    c, p = strongly_entangling(6, 1, seed=3)
    sv = StateVector(6, "c128")
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    E, _ = prog.jacobian()
    _assert_rel(E.cpu().numpy(), oracle.adjoint_jacobian(c, p)[0], TOL_E["c128"], "expvals", "c128")
    sv.close()
    assert sv.handle is None and prog.handle is None
    prog.close()  # already closed: a no-op
    with pytest.raises(RuntimeError):
        Program.from_circuit(sv, c)
