"""The 30-qubit stress workload at full size: 20 layers of RY on all wires plus
a CZ brick, with a seeded 5-qubit dense block after every fifth layer (tensor
cores in complex64, CUDA cores in complex128), observable Z_0 Z_29, forward
pass plus full adjoint Jacobian (600 parameters), complex128 (16 GiB per
vector) and complex64.

Checks (bars as in tests/bars.py):
  * the FP64 oracle's <Z_0 Z_29> and full 600-entry Jacobian at n = 30 by its
    adjoint method, stored in tests/golden/rycz30_jacobian.txt by
    tests/golden/make_rycz30_jacobian.py, which calls only the oracle (three
    16 GiB vectors, one to two hours of CPU time), element by element in
    complex128 and complex64;
  * the oracle's <Z_0 Z_29> from a forward pass alone
    (tests/golden/rycz30_expval.txt, tests/golden/make_rycz30_expval.py);
  * parameter shift with the GPU's own forward passes on a seeded sample of
    parameters: every RY has G = Y with eigenvalues +-1, so
    dE/dtheta = (E(theta + pi/2) - E(theta - pi/2)) / 2 exactly;
  * complex64 against complex128.
"""

import os

import numpy as np
import pytest

import bars
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
    floor = bars.FLOOR * float(np.abs(J).max())
    for q, g in shift.items():
        assert abs(J[0, q] - g) <= 1e-9 * max(abs(g), floor), (q, J[0, q], g)


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
    bars.check_e([float(E[0])], E128, "c64", "rycz30 c64 vs c128 expval")
    bars.check_j(J.cpu().numpy(), J128, "c64", "rycz30 c64 vs c128 jacobian")
    golden = _golden_jacobian()
    if golden is not None:
        Eo, Jo = golden
        bars.record("rycz30 expval vs oracle", "c64", E.cpu().numpy(), [Eo],
                    bars.check_e(E.cpu().numpy(), [Eo], "c64", "rycz30 expval vs oracle"))
        bars.record("rycz30 jacobian vs oracle", "c64", J.cpu().numpy()[0], Jo,
                    bars.check_j(J.cpu().numpy()[0], Jo, "c64", "rycz30 jacobian vs oracle"))


def _golden_expval() -> float:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rycz30_expval.txt")
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            return float(ln)
    raise ValueError("no value in " + path)


def _golden_jacobian():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rycz30_jacobian.txt")
    if not os.path.exists(path):
        return None
    vals = [float(ln) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(vals) == 601, path
    return vals[0], np.array(vals[1:])


def test_rycz30_c128_expval_matches_oracle(c128_result):
    # the FP64 oracle's value at n = 30, written by tests/golden/make_rycz30_expval.py
    want = _golden_expval()
    E128 = c128_result[0]
    bars.record("rycz30 expval vs oracle forward", "c128", E128, [want],
                bars.check_e(E128, [want], "c128", "rycz30 expval vs oracle forward"))


def test_rycz30_c128_jacobian_matches_oracle(c128_result):
    # the FP64 oracle's adjoint Jacobian at n = 30, written by tests/golden/make_rycz30_jacobian.py
    golden = _golden_jacobian()
    assert golden is not None, "tests/golden/rycz30_jacobian.txt is missing"
    Eo, Jo = golden
    E, J, _ = c128_result
    bars.record("rycz30 expval vs oracle", "c128", E, [Eo], bars.check_e(E, [Eo], "c128", "rycz30 expval vs oracle"))
    bars.record("rycz30 jacobian vs oracle", "c128", J[0], Jo,
                bars.check_j(J[0], Jo, "c128", "rycz30 jacobian vs oracle"))
