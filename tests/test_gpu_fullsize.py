"""The workloads at their benchmark sizes against the FP64 oracle.

* sel24: 24-qubit strongly-entangling layers (8 layers of Rot per wire plus a
  CNOT ring of range l mod 23 + 1), 24 single-Z observables: expectation
  values and the full 24 x 576 adjoint Jacobian, element by element, in the
  launch configuration the benchmark times (planned program, parameters on
  the device), in complex128, double-float and complex64.
* VQE-24: Hartree-Fock start, 120 DoubleExcitation + 40 SingleExcitation
  gates, a Hamiltonian of 2000 Pauli words of weight 2-4: energy and the
  160-entry gradient (the many-word expectation and lambda kernels).
* QAOA MaxCut batches: 512 parameter sets of the 20-node p = 4 circuit and
  256 mixed 14-22-qubit instances in one persistent launch, run as several
  L2 waves (the benchmark's schedule), a seeded sample of circuits from every
  part of the schedule against the oracle.

Bars as in tests/bars.py (complex128 1e-10 / 1e-9 entry-wise relative with a
1e-3 floor, complex64 1e-4 normwise).
"""

import numpy as np
import pytest

import bars
import oracle
from workloads import qaoa_maxcut, qaoa_mixed_instances, qaoa_param_sets, strongly_entangling, vqe_givens

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - GPU-only module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_02512_gb300 import _lib as L  # noqa: E402
from paper_2403_02512_gb300.torch_api import Program, StateVector  # noqa: E402

DTYPES = ["c128", "c128df", "c64"]


@pytest.fixture(scope="module")
def sel24():
    c, p = strongly_entangling(24, 8)
    Eo, Jo = oracle.adjoint_jacobian(c, p)
    return c, p, Eo, Jo


def _bench_step(c, p, dtype):
    """Forward pass + expectation values + adjoint Jacobian exactly as the
    benchmark launches them (parameters set from a device tensor)."""
    sv = StateVector(c.n, dtype, basis_state=c.basis_state)
    prog = Program.from_circuit(sv, c)
    params = torch.tensor(p, dtype=torch.float64, device="cuda")
    prog.set_params(params)
    prog.forward()
    E, J = prog.jacobian()
    out = E.cpu().numpy(), J.cpu().numpy()
    prog.close()
    sv.close()
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("dtype", DTYPES)
def test_sel24_jacobian_full_size(sel24, dtype):
    c, p, Eo, Jo = sel24
    E, J = _bench_step(c, p, dtype)
    assert J.shape == (24, 576)
    bars.record("sel24 expvals", dtype, E, Eo, bars.check_e(E, Eo, dtype, "sel24 expvals"))
    bars.record("sel24 jacobian", dtype, J, Jo, bars.check_j(J, Jo, dtype, "sel24 jacobian"))


@pytest.fixture(scope="module")
def vqe24():
    c, p = vqe_givens(24, 12, 40, 120, 2000)
    Eo, Jo = oracle.adjoint_jacobian(c, p)
    return c, p, Eo, Jo


@pytest.mark.parametrize("dtype", DTYPES)
def test_vqe24_2000_words_full_size(vqe24, dtype):
    c, p, Eo, Jo = vqe24
    assert len(c.observables[0]) == 2000 and c.n_params == 160
    E, J = _bench_step(c, p, dtype)
    bars.record("vqe24 energy", dtype, E, Eo, bars.check_e(E, Eo, dtype, "vqe24 energy"))
    bars.record("vqe24 gradient", dtype, J, Jo, bars.check_j(J, Jo, dtype, "vqe24 gradient"))
    # the energy-and-gradient step of the benchmark: expectation value, then one
    # lambda = H phi swept backwards (VJP with weight 1)
    sv = StateVector(c.n, dtype, basis_state=c.basis_state)
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    e = prog.expval().cpu().numpy()
    g = prog.vjp(np.ones(1)).cpu().numpy()
    prog.close()
    sv.close()
    bars.record("vqe24 energy (expval call)", dtype, e, Eo, bars.check_e(e, Eo, dtype, "vqe24 energy (expval call)"))
    bars.record("vqe24 gradient (vjp)", dtype, g, Jo[0], bars.check_j(g, Jo[0], dtype, "vqe24 gradient (vjp)"))


def _sample(count, k, seed):
    """k indices spread over the whole batch: the first, the last and a seeded rest."""
    rng = np.random.default_rng(seed)
    rest = rng.choice(np.arange(1, count - 1), size=k - 2, replace=False)
    return np.unique(np.concatenate([[0, count - 1], rest]))


def _oracle_energy(c, p):
    return oracle.expval(oracle.forward(c, p), c.observables[0])


@pytest.mark.parametrize("dtype,tuned", [(L.SV_C64, False), (L.SV_C64, True), (L.SV_C128, False)])
def test_qaoa20_x512_batch_multi_wave(dtype, tuned):
    c = qaoa_maxcut(20, 4)
    sets = qaoa_param_sets(512, 4)
    b = L.Batch([c] * len(sets), dtype)
    b.set_params(sets.ravel())
    if tuned:
        b.autotune()
    got = b.run()
    info = b.info()
    amp = 8 if dtype == L.SV_C64 else 16
    assert info["wave_bytes"] < len(sets) * (amp << 20), "the schedule must run several waves"
    idx = _sample(len(sets), 32, 512)
    want = np.array([_oracle_energy(c, sets[i]) for i in idx])
    name = "c64" if dtype == L.SV_C64 else "c128"
    what = f"qaoa20 x512 batch{' (autotuned)' if tuned else ''}"
    bars.record(what, name, got[idx], want, bars.check_e(got[idx], want, name, what))
    again = b.run()  # graph replay: bitwise the same
    assert np.array_equal(got, again)
    b.close()
    torch.cuda.empty_cache()


def test_qaoa_mixed_14_to_22_x256_batch_multi_wave():
    inst = qaoa_mixed_instances(256, 14, 22, 4)
    b = L.Batch([ci for ci, _ in inst], L.SV_C64)
    b.set_params(np.concatenate([pi for _, pi in inst]))
    b.autotune()
    got = b.run()
    total = sum(8 << ci.n for ci, _ in inst)
    assert b.info()["wave_bytes"] < total, "the schedule must run several waves"
    sizes = np.array([ci.n for ci, _ in inst])
    idx = set(_sample(len(inst), 24, 256).tolist())
    idx |= {int(np.argmax(sizes)), int(np.argmin(sizes))}  # the largest and smallest instances
    idx = sorted(idx)
    want = np.array([_oracle_energy(*inst[i]) for i in idx])
    bars.record("qaoa mixed 14-22 x256 batch", "c64", got[idx], want,
                bars.check_e(got[idx], want, "c64", "qaoa mixed 14-22 x256 batch"))
    b.close()
    torch.cuda.empty_cache()
