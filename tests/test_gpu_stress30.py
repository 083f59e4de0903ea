"""The 30-qubit stress workload at full size: 20 layers of RY on all wires plus
a CZ brick, with a seeded 5-qubit dense block after every fifth layer (tensor
cores in complex64, CUDA cores in complex128), observable Z_0 Z_29, forward
pass plus full adjoint Jacobian (600 parameters), complex128 (16 GiB per
vector) and complex64.

No dense reference exists at this size, so the checks are:
  * parameter shift, computed with the GPU's own forward passes, on a seeded
    sample of parameters: every RY has G = Y with eigenvalues +-1, so
    dE/dtheta = (E(theta + pi/2) - E(theta - pi/2)) / 2 exactly (complex128 bar
    1e-9 relative to max(1, max|J|));
  * the FP64 oracle's <Z_0 Z_29> at n = 30 (complex128 bar 1e-10), stored in
    tests/golden/rycz30_expval.txt by tests/golden/make_rycz30_expval.py, which
    calls only the oracle (two 16 GiB vectors, minutes of CPU time);
  * complex64 against complex128 (complex64 bar 1e-4).
"""

import os

import numpy as np
import pytest

from workloads import config_seed, ry_cz_brick

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - GPU-only module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_02512_gb300.torch_api import Program, StateVector  # noqa: E402

N = 30


@pytest.fixture(scope="module")
def workload():
    c, p = ry_cz_brick(N, 20)
    assert sum(op.name == "QubitUnitary" for op in c.ops) == 4
    return c, p


@pytest.fixture(scope="module")
def c128_result(workload):
    c, p = workload
    sv = StateVector(N, "c128")
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    E, J = prog.jacobian()
    E, J = E.cpu().numpy(), J.cpu().numpy()
    # parameter shift on a seeded sample of parameters, GPU forward passes
    rng = np.random.default_rng(config_seed(5) + 1)
    sample = rng.choice(c.n_params, 8, replace=False)
    shift = {}
    for q in sample:
        e = []
        for d in (0.5 * np.pi, -0.5 * np.pi):
            pp = p.copy()
            pp[q] += d
            prog.forward(pp)
            e.append(float(prog.expval()[0]))
        shift[int(q)] = 0.5 * (e[0] - e[1])
    prog.close()
    sv.close()
    torch.cuda.empty_cache()
    return E, J, shift


def test_rycz30_c128_jacobian_matches_parameter_shift(c128_result):
    E, J, shift = c128_result
    assert J.shape == (1, 600) and np.all(np.isfinite(J))
    scale = max(1.0, float(np.abs(J).max()))
    for q, g in shift.items():
        assert abs(J[0, q] - g) <= 1e-9 * scale, (q, J[0, q], g)


def test_rycz30_c64_matches_c128(workload, c128_result):
    c, p = workload
    E128, J128, _ = c128_result
    sv = StateVector(N, "c64")
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    E, J = prog.jacobian()
    prog.close()
    sv.close()
    torch.cuda.empty_cache()
    assert abs(float(E[0]) - float(E128[0])) <= 1e-4
    assert float(np.abs(J.cpu().numpy() - J128).max()) <= 1e-4 * max(1.0, float(np.abs(J128).max()))


def _golden_expval() -> float:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rycz30_expval.txt")
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            return float(ln)
    raise ValueError("no value in " + path)


def test_rycz30_c128_expval_matches_oracle(c128_result):
    # the FP64 oracle's value at n = 30, written by tests/golden/make_rycz30_expval.py
    want = _golden_expval()
    E128 = c128_result[0]
    assert abs(float(E128[0]) - want) <= 1e-10 * max(1.0, abs(want))
