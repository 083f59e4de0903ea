"""sv_expval_static: expectation values with no device allocation.

Callers that cannot allocate device memory when they measure (a process that
reserved all GPU memory up front, code where cudaMalloc / cudaFree and the
synchronisation of cudaFree are not allowed) use this entry point; it keeps
every temporary in a fixed array compiled into the library.  These tests call
it through the C ABI and check it against sv_expval, the allocating entry
point, on two calls in a row (the array keeps the previous call's contents,
so the second call shows that nothing stale leaks into it).

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

from workloads import Term, random_hamiltonian, random_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - GPU-only module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_02512_gb300 import _lib as L  # noqa: E402
from paper_2403_02512_gb300.torch_api import StateVector  # noqa: E402

TOL = {"c128": 1e-10, "c64": 1e-4}


def _observables(n, seed, n_obs=4, n_terms=60):
    rng = np.random.default_rng(seed)
    obs = [random_hamiltonian(n, n_terms, rng, weights=tuple(range(1, min(n, 4) + 1))) for _ in range(n_obs)]
    obs.append([Term(0.25, ())])                       # identity term
    obs.append([])                                      # no terms
    return obs


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [3, 13, 18])
def test_static_expval_matches_allocating_expval_twice(dtype, n):
    for call, seed in enumerate((n, n + 100)):
        sv = StateVector(n, dtype)
        sv.set_numpy(random_state(n, seed))
        obs = _observables(n, seed)
        ps = L.PauliSums(obs)
        want = L.sv_expval(sv.handle, ps)
        torch.cuda.synchronize()
        got = L.sv_expval_static(sv.tensor.data_ptr(), n, sv.sv_dtype, ps,
                                 torch.cuda.current_stream().cuda_stream)
        scale = np.maximum(1.0, np.abs(want))
        assert np.all(np.abs(got - want) <= TOL[dtype] * scale), (call, got, want)
        sv.close()


def test_static_expval_rejects_sizes_beyond_its_limits():
    sv = StateVector(4, "c128")
    too_many = [[Term(1.0, ((0, "Z"),))] * 5000]
    with pytest.raises(L.SvError) as ei:
        L.sv_expval_static(sv.tensor.data_ptr(), 4, sv.sv_dtype, L.PauliSums(too_many))
    assert ei.value.status == 1 and "SV_STATIC_MAX_TERMS" in str(ei.value)
    too_many_obs = [[Term(1.0, ((0, "Z"),))]] * 1025
    with pytest.raises(L.SvError) as ei:
        L.sv_expval_static(sv.tensor.data_ptr(), 4, sv.sv_dtype, L.PauliSums(too_many_obs))
    assert ei.value.status == 1 and "SV_STATIC_MAX_OBSERVABLES" in str(ei.value)
