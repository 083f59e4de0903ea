"""sv_expval_static: expectation values with no device allocation.

Callers that cannot allocate device memory when they measure (a process that
reserved all GPU memory up front, code where cudaMalloc / cudaFree and the
synchronisation of cudaFree are not allowed) use this entry point; it keeps
every temporary in a fixed array compiled into the library.  These tests call
it through the C ABI and check it against the FP64 oracle and against
sv_expval, the allocating entry point, on two calls in a row (the array keeps
the previous call's contents, so the second call shows that nothing stale
leaks into it); that a call leaves the device's free memory unchanged; and
that bad pointers and sizes beyond its limits are rejected before any launch.

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

import bars
import oracle
from workloads import Term, random_hamiltonian, random_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - GPU-only module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_02512_gb300 import _lib as L  # noqa: E402
from paper_2403_02512_gb300.torch_api import StateVector  # noqa: E402


def _observables(n, seed, n_obs=4, n_terms=60):
    rng = np.random.default_rng(seed)
    obs = [random_hamiltonian(n, n_terms, rng, weights=tuple(range(1, min(n, 4) + 1))) for _ in range(n_obs)]
    obs.append([Term(0.25, ())])                       # identity term
    obs.append([])                                      # no terms
    return obs


def _static(sv, n, ps):
    return L.sv_expval_static(sv.tensor.data_ptr(), n, sv.sv_dtype, ps, torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [3, 13, 18])
def test_static_expval_matches_oracle_and_allocating_expval_twice(dtype, n):
    for call, seed in enumerate((n, n + 100)):
        sv = StateVector(n, dtype)
        sv.set_numpy(random_state(n, seed))
        psi = sv.to_numpy().astype(np.complex128)  # the oracle reads exactly the amplitudes the GPU holds
        obs = _observables(n, seed)
        ps = L.PauliSums(obs)
        want = L.sv_expval(sv.handle, ps)
        torch.cuda.synchronize()
        got = _static(sv, n, ps)
        bars.check_e(got, want, dtype, f"static vs sv_expval, call {call}")
        bars.check_e(got, np.array([oracle.expval(psi, H) for H in obs]), dtype, f"static vs oracle, call {call}")
        sv.close()


def test_static_expval_allocates_nothing():
    n = 16
    sv = StateVector(n, "c128")
    sv.set_numpy(random_state(n, 5))
    small = L.PauliSums(_observables(n, 5, n_obs=1, n_terms=4))
    large = L.PauliSums(_observables(n, 6, n_obs=200, n_terms=20))  # 4000 terms, 202 observables
    _static(sv, n, small)  # first call on the device: looks up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for ps in (large, small, large):
        _static(sv, n, ps)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_expval_empty_observables_give_zeros():
    n = 7
    sv = StateVector(n, "c64")
    sv.set_numpy(random_state(n, 9))
    got = _static(sv, n, L.PauliSums([[], [], []]))
    assert np.array_equal(got, np.zeros(3))


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


def test_static_expval_rejects_a_word_flipping_more_wires_than_a_tile():
    n = 16
    sv = StateVector(n, "c128")
    wide = [[Term(1.0, tuple((w, "X") for w in range(n)))]]  # flips all 16 wires; a tile holds 11
    with pytest.raises(L.SvError) as ei:
        _static(sv, n, L.PauliSums(wide))
    assert ei.value.status == 5


def test_static_expval_rejects_memory_it_cannot_read():
    ps = L.PauliSums([[Term(1.0, ((0, "Z"),))]])
    host = np.zeros(1 << 10, dtype=np.complex128)
    with pytest.raises(L.SvError) as ei:  # pageable host memory
        L.sv_expval_static(host.ctypes.data, 10, L.SV_C128, ps)
    assert ei.value.status == 1
    pinned = torch.zeros(1 << 10, dtype=torch.complex128).pin_memory()
    with pytest.raises(L.SvError) as ei:  # pinned host memory
        L.sv_expval_static(pinned.data_ptr(), 10, L.SV_C128, ps)
    assert ei.value.status == 1
    small = torch.zeros(1 << 10, dtype=torch.complex128, device="cuda")
    with pytest.raises(L.SvError) as ei:  # 2^30 amplitudes claimed on a 16 KiB tensor
        L.sv_expval_static(small.data_ptr(), 30, L.SV_C128, ps)
    assert ei.value.status == 1 and "fewer than 2^n" in str(ei.value)
