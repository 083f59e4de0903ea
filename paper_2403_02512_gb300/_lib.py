"""ctypes binding of ``libsv.so`` (the C ABI declared in include/sv.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Functions keep the C names (``sv_create``, ``sv_apply``, ...), take
Python / numpy arguments and raise :class:`SvError` on a non-zero status.
There is no CPU fallback: if the library cannot be built or loaded, every
call raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import NamedTuple, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsv.so")

SV_MAX_TARGETS = 6
SV_MAX_CONTROLS = 8
SV_MAX_QUBITS = 34

SV_C64, SV_C128 = 0, 1
SV_COMPUTE_NATIVE, SV_COMPUTE_DOUBLE_FLOAT = 0, 1

STATUS = {0: "SV_OK", 1: "SV_ERR_ARG", 2: "SV_ERR_OOM", 3: "SV_ERR_CUDA", 4: "SV_ERR_TIMEOUT",
          5: "SV_ERR_UNSUPPORTED", 6: "SV_ERR_STATE"}

KIND = {
    "Identity": 0, "PauliX": 1, "PauliY": 2, "PauliZ": 3, "Hadamard": 4, "S": 5, "T": 6,
    "PhaseShift": 7, "RX": 8, "RY": 9, "RZ": 10, "Rot": 11, "SWAP": 12, "IsingXX": 13,
    "IsingYY": 14, "IsingZZ": 15, "IsingXY": 16, "SingleExcitation": 17,
    "DoubleExcitation": 18, "QubitUnitary": 19,
}


class SvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class SvOp(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n_targets", ctypes.c_int32),
        ("targets", ctypes.c_int32 * SV_MAX_TARGETS),
        ("n_controls", ctypes.c_int32),
        ("controls", ctypes.c_int32 * SV_MAX_CONTROLS),
        ("control_values", ctypes.c_int32 * SV_MAX_CONTROLS),
        ("param_index", ctypes.c_int32 * 3),
        ("const_angle", ctypes.c_double * 3),
        ("scale", ctypes.c_double),
        ("adjoint", ctypes.c_int32),
        ("matrix_offset", ctypes.c_int64),
    ]


class SvTape(ctypes.Structure):
    _fields_ = [
        ("n_ops", ctypes.c_int32),
        ("ops", ctypes.POINTER(SvOp)),
        ("n_params", ctypes.c_int32),
        ("matrices", ctypes.POINTER(ctypes.c_double)),
        ("n_matrix_entries", ctypes.c_int64),
    ]


class SvPauliSum(ctypes.Structure):
    _fields_ = [
        ("n_terms", ctypes.c_int32),
        ("coeffs", ctypes.POINTER(ctypes.c_double)),
        ("x_mask", ctypes.POINTER(ctypes.c_uint64)),
        ("z_mask", ctypes.POINTER(ctypes.c_uint64)),
    ]


# exported symbols and their prototypes: (restype, argtypes)
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
PROTOTYPES = {
    "sv_last_error": (ctypes.c_char_p, []),
    "sv_version": (ctypes.c_char_p, []),
    "sv_set_alloc_cap": (ctypes.c_int, [ctypes.c_size_t]),
    "sv_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "sv_create_from_device_ptr": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "sv_destroy": (ctypes.c_int, [_vp]),
    "sv_set_stream": (ctypes.c_int, [_vp, _vp]),
    "sv_set_workspace": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "sv_info": (ctypes.c_int, [_vp, _ip, _ip, ctypes.POINTER(_vp)]),
    "sv_set_compute": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sv_set_renormalize": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sv_set_dense_tensor_cores": (ctypes.c_int, [ctypes.c_int]),
    "sv_reset": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "sv_set_state": (ctypes.c_int, [_vp, _vp]),
    "sv_get_state": (ctypes.c_int, [_vp, _vp]),
    "sv_synchronize": (ctypes.c_int, [_vp]),
    "sv_apply": (ctypes.c_int, [_vp, ctypes.c_int, _ip, ctypes.c_int, _dp, ctypes.c_int]),
    "sv_apply_op": (ctypes.c_int, [_vp, ctypes.POINTER(SvOp), _dp, _dp]),
    "sv_apply_matrix": (ctypes.c_int, [_vp, _ip, ctypes.c_int, _dp, ctypes.c_int]),
    "sv_expval": (ctypes.c_int, [_vp, ctypes.POINTER(SvPauliSum), ctypes.c_int, _dp]),
    "sv_norm2": (ctypes.c_int, [_vp, _dp]),
    "sv_var": (ctypes.c_int, [_vp, ctypes.POINTER(SvPauliSum), ctypes.c_int, _dp]),
    "sv_probs": (ctypes.c_int, [_vp, _ip, ctypes.c_int, _dp]),
    "sv_sample": (ctypes.c_int, [_vp, _ip, ctypes.c_int, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]),
    "sv_forward": (ctypes.c_int, [_vp, ctypes.POINTER(SvTape), _dp]),
    "sv_adjoint_jacobian": (ctypes.c_int, [_vp, ctypes.POINTER(SvTape), _dp, ctypes.POINTER(SvPauliSum),
                                           ctypes.c_int, _dp, _dp]),
    "sv_adjoint_vjp": (ctypes.c_int, [_vp, ctypes.POINTER(SvTape), _dp, ctypes.POINTER(SvPauliSum),
                                      ctypes.c_int, _dp, _dp]),
    "sv_program_create": (ctypes.c_int, [_vp, ctypes.POINTER(SvTape), ctypes.POINTER(SvPauliSum),
                                         ctypes.c_int, ctypes.POINTER(_vp)]),
    "sv_program_destroy": (ctypes.c_int, [_vp]),
    "sv_program_set_params": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "sv_program_forward": (ctypes.c_int, [_vp]),
    "sv_program_jacobian": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "sv_program_expval": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "sv_program_vjp": (ctypes.c_int, [_vp, _dp, _vp, ctypes.c_int]),
    "sv_program_jvp": (ctypes.c_int, [_vp, _dp, _vp, ctypes.c_int]),
    "sv_sparse_create": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _dp, ctypes.c_int64, ctypes.POINTER(_vp)]),
    "sv_sparse_destroy": (ctypes.c_int, [_vp]),
    "sv_sparse_expval": (ctypes.c_int, [_vp, _vp, _dp]),
    "sv_adjoint_jacobian_sparse": (ctypes.c_int, [_vp, ctypes.POINTER(SvTape), _dp, _vp, _dp, _dp]),
    "sv_program_stats": (ctypes.c_int, [_vp, _ip, _ip, _ip]),
    "sv_plan_query": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(SvTape), _ip, _ip]),
    "sv_plan_describe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(SvTape), _ip, _ip]),
    "sv_hermitian_to_pauli": (ctypes.c_int, [ctypes.c_int, _ip, ctypes.c_int, _dp, ctypes.c_double, _dp,
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _ip]),
    "sv_kernel_timing_enable": (ctypes.c_int, [ctypes.c_int]),
    "sv_kernel_timing_reset": (ctypes.c_int, []),
    "sv_kernel_timing_read": (ctypes.c_int, [_dp, ctypes.POINTER(ctypes.c_int64)]),
    "sv_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _ip, ctypes.POINTER(SvTape),
                                       ctypes.POINTER(SvPauliSum), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(_vp)]),
    "sv_batch_destroy": (ctypes.c_int, [_vp]),
    "sv_batch_set_stream": (ctypes.c_int, [_vp, _vp]),
    "sv_batch_set_params": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "sv_batch_run": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "sv_batch_status": (ctypes.c_int, [_vp]),
    "sv_batch_autotune": (ctypes.c_int, [_vp, _dp]),
    "sv_batch_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), _ip, _ip, ctypes.POINTER(ctypes.c_int64),
                                     _ip]),
    "sv_expval_static": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(SvPauliSum), ctypes.c_int,
                                        _dp, _vp]),
}

KERNEL_CLASSES = ["tile_forward", "tile_adjoint", "expval", "lambda", "reduce", "build_matrices", "dense_k",
                  "other"]

_LIB: Optional[ctypes.CDLL] = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsv.so (building it with nvcc first if it is absent or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsv.so not found at {LIB_PATH}; build it with paper_2403_02512_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _check(status: int) -> None:
    if status != 0:
        msg = load().sv_last_error()
        raise SvError(status, msg.decode() if msg else "")


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _iarr(xs: Sequence[int]):
    return (ctypes.c_int * max(1, len(xs)))(*[int(x) for x in xs])


# ---------------------------------------------------------------------------
# Thin wrappers with the C names
# ---------------------------------------------------------------------------
def sv_version() -> str:
    return load().sv_version().decode()


def sv_set_alloc_cap(nbytes: int) -> None:
    _check(load().sv_set_alloc_cap(int(nbytes)))


def sv_create(n: int, dtype: int) -> int:
    h = _vp()
    _check(load().sv_create(int(n), int(dtype), ctypes.byref(h)))
    return h.value


def sv_create_from_device_ptr(n: int, dtype: int, device_ptr: int) -> int:
    h = _vp()
    _check(load().sv_create_from_device_ptr(int(n), int(dtype), _vp(device_ptr), ctypes.byref(h)))
    return h.value


def sv_destroy(h: int) -> None:
    _check(load().sv_destroy(_vp(h)))


def sv_set_stream(h: int, stream: int) -> None:
    _check(load().sv_set_stream(_vp(h), _vp(stream)))


def sv_set_workspace(h: int, device_ptr: int, nbytes: int) -> None:
    _check(load().sv_set_workspace(_vp(h), _vp(device_ptr), int(nbytes)))


def sv_set_compute(h: int, compute: int) -> None:
    _check(load().sv_set_compute(_vp(h), int(compute)))


def sv_set_renormalize(h: int, on: bool) -> None:
    _check(load().sv_set_renormalize(_vp(h), 1 if on else 0))


def sv_set_dense_tensor_cores(on: bool) -> None:
    _check(load().sv_set_dense_tensor_cores(1 if on else 0))


def sv_info(h: int):
    n, dt, ptr = ctypes.c_int(), ctypes.c_int(), _vp()
    _check(load().sv_info(_vp(h), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(ptr)))
    return n.value, dt.value, ptr.value


def sv_reset(h: int, basis_index: int = 0) -> None:
    _check(load().sv_reset(_vp(h), int(basis_index)))


def sv_set_state(h: int, host: np.ndarray) -> None:
    assert host.flags["C_CONTIGUOUS"]
    _check(load().sv_set_state(_vp(h), host.ctypes.data_as(_vp)))


def sv_get_state(h: int, out: np.ndarray) -> np.ndarray:
    assert out.flags["C_CONTIGUOUS"]
    _check(load().sv_get_state(_vp(h), out.ctypes.data_as(_vp)))
    return out


def sv_synchronize(h: int) -> None:
    _check(load().sv_synchronize(_vp(h)))


def sv_apply(h: int, kind: int, wires: Sequence[int], angles: Optional[Sequence[float]] = None,
             adjoint: bool = False) -> None:
    a = None if angles is None or len(angles) == 0 else np.ascontiguousarray(angles, dtype=np.float64)
    _check(load().sv_apply(_vp(h), int(kind), _iarr(wires), len(wires), _dptr(a), int(bool(adjoint))))


def sv_apply_op(h: int, op: SvOp, params: Optional[np.ndarray] = None, matrices: Optional[np.ndarray] = None):
    _check(load().sv_apply_op(_vp(h), ctypes.byref(op), _dptr(params), _dptr(matrices)))


def sv_apply_matrix(h: int, wires: Sequence[int], matrix: np.ndarray, adjoint: bool = False) -> None:
    m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128)).view(np.float64).ravel()
    k = len(wires)
    assert m.size == 2 * (1 << (2 * k))
    _check(load().sv_apply_matrix(_vp(h), _iarr(wires), k, _dptr(m), int(bool(adjoint))))


def sv_expval(h: int, obs: "PauliSums") -> np.ndarray:
    out = np.zeros(obs.count, dtype=np.float64)
    _check(load().sv_expval(_vp(h), obs.array, obs.count, _dptr(out)))
    return out


def sv_var(h: int, obs: "PauliSums") -> np.ndarray:
    out = np.zeros(obs.count, dtype=np.float64)
    _check(load().sv_var(_vp(h), obs.array, obs.count, _dptr(out)))
    return out


def _wires(wires):
    arr = (ctypes.c_int * max(1, len(wires)))(*[int(w) for w in wires])
    return arr, len(wires)


def sv_probs(h: int, wires) -> np.ndarray:
    arr, k = _wires(wires)
    out = np.zeros(1 << k, dtype=np.float64)
    _check(load().sv_probs(_vp(h), arr, k, _dptr(out)))
    return out


def sv_sample(h: int, wires, uniforms) -> np.ndarray:
    arr, k = _wires(wires)
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    out = np.zeros(u.size, dtype=np.uint64)
    _check(load().sv_sample(_vp(h), arr, k, _dptr(u), u.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return out


def sv_norm2(h: int) -> float:
    out = np.zeros(1)
    _check(load().sv_norm2(_vp(h), _dptr(out)))
    return float(out[0])


def sv_forward(h: int, tape: "Tape", params: np.ndarray) -> None:
    p = np.ascontiguousarray(params, dtype=np.float64)
    _check(load().sv_forward(_vp(h), ctypes.byref(tape.struct), _dptr(p)))


def sv_adjoint_jacobian(h: int, tape: "Tape", params: np.ndarray, obs: "PauliSums"):
    p = np.ascontiguousarray(params, dtype=np.float64)
    E = np.zeros(obs.count)
    J = np.zeros((obs.count, tape.n_params))
    _check(load().sv_adjoint_jacobian(_vp(h), ctypes.byref(tape.struct), _dptr(p), obs.array, obs.count,
                                      _dptr(E), _dptr(J)))
    return E, J


def sv_adjoint_vjp(h: int, tape: "Tape", params: np.ndarray, obs: "PauliSums", grad_out) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    g = np.ascontiguousarray(grad_out, dtype=np.float64)
    out = np.zeros(tape.n_params)
    _check(load().sv_adjoint_vjp(_vp(h), ctypes.byref(tape.struct), _dptr(p), obs.array, obs.count, _dptr(g),
                                 _dptr(out)))
    return out


def sv_program_create(h: int, tape: "Tape", obs: Optional["PauliSums"]) -> int:
    ph = _vp()
    arr = obs.array if obs is not None else None
    cnt = obs.count if obs is not None else 0
    _check(load().sv_program_create(_vp(h), ctypes.byref(tape.struct), arr, cnt, ctypes.byref(ph)))
    return ph.value


def sv_program_destroy(ph: int) -> None:
    _check(load().sv_program_destroy(_vp(ph)))


def sv_program_set_params(ph: int, params_ptr: int, on_device: bool) -> None:
    _check(load().sv_program_set_params(_vp(ph), _vp(params_ptr), int(on_device)))


def sv_program_forward(ph: int) -> None:
    _check(load().sv_program_forward(_vp(ph)))


def sv_program_jacobian(ph: int, expvals_ptr: int, jac_ptr: int, on_device: bool) -> None:
    _check(load().sv_program_jacobian(_vp(ph), _vp(expvals_ptr), _vp(jac_ptr), int(on_device)))


def sv_program_expval(ph: int, expvals_ptr: int, on_device: bool) -> None:
    _check(load().sv_program_expval(_vp(ph), _vp(expvals_ptr), int(on_device)))


def sv_program_vjp(ph: int, grad_out: np.ndarray, vjp_ptr: int, on_device: bool) -> None:
    g = np.ascontiguousarray(grad_out, dtype=np.float64)
    _check(load().sv_program_vjp(_vp(ph), _dptr(g), _vp(vjp_ptr), int(on_device)))


def sv_program_jvp(ph: int, tangent: np.ndarray, out_ptr: int, on_device: bool) -> None:
    t = np.ascontiguousarray(tangent, dtype=np.float64)
    _check(load().sv_program_jvp(_vp(ph), _dptr(t), _vp(out_ptr), int(on_device)))


class Sparse:
    """A CSR observable on the device (sv_sparse_create / sv_sparse_destroy)."""

    def __init__(self, n: int, indptr, indices, values):
        self.n = int(n)
        ip = np.ascontiguousarray(indptr, dtype=np.int64)
        ix = np.ascontiguousarray(indices, dtype=np.int64)
        v = np.ascontiguousarray(np.asarray(values, dtype=np.complex128).view(np.float64))
        h = _vp()
        _check(load().sv_sparse_create(self.n, ip.ctypes.data, ix.ctypes.data if ix.size else None,
                                       _dptr(v) if v.size else None, ix.size, ctypes.byref(h)))
        self.handle = h.value

    def close(self) -> None:
        if getattr(self, "handle", None):
            load().sv_sparse_destroy(_vp(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sv_sparse_expval(h: int, sp: Sparse) -> float:
    out = np.zeros(1)
    _check(load().sv_sparse_expval(_vp(h), _vp(sp.handle), _dptr(out)))
    return float(out[0])


def sv_adjoint_jacobian_sparse(h: int, tape: "Tape", params, sp: Sparse):
    p = np.ascontiguousarray(params, dtype=np.float64)
    e = np.zeros(1)
    J = np.zeros(max(1, tape.n_params))
    _check(load().sv_adjoint_jacobian_sparse(_vp(h), ctypes.byref(tape.struct), _dptr(p) if p.size else None,
                                             _vp(sp.handle), _dptr(e), _dptr(J)))
    return float(e[0]), J[: tape.n_params]


PLAN_KINDS = ("pair", "diag", "dense", "phase_run", "fused_run", "multi", "wide_dense", "passes")


def sv_plan_describe(n: int, dtype: int, tape: "Tape"):
    """Micro-op counts of the forward and adjoint plans (host only)."""
    f = (ctypes.c_int * 8)()
    a = (ctypes.c_int * 8)()
    _check(load().sv_plan_describe(int(n), int(dtype), ctypes.byref(tape.struct), f, a))
    return dict(zip(PLAN_KINDS, list(f))), dict(zip(PLAN_KINDS, list(a)))


SV_MAX_HERMITIAN_WIRES = 5


class PauliTerm(NamedTuple):
    """One word of a Hamiltonian: coeff * prod over (wire, letter) of the Pauli letter."""
    coeff: float
    paulis: Tuple[Tuple[int, str], ...]


def sv_hermitian_to_pauli(n: int, wires, matrix, tol: float = 0.0):
    """The Pauli words of a Hermitian matrix on ``wires`` (host only): a list of
    PauliTerm usable wherever a Hamiltonian (list of terms) is accepted."""
    w = np.ascontiguousarray(list(wires), dtype=np.int32)
    k = int(w.size)
    m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
    if k < 1 or m.shape != (1 << k, 1 << k):
        raise SvError(1, "matrix must be 2^k x 2^k for k wires")
    cap = 1 << (2 * k)
    c = np.zeros(cap, dtype=np.float64)
    x = np.zeros(cap, dtype=np.uint64)
    z = np.zeros(cap, dtype=np.uint64)
    cnt = ctypes.c_int()
    _check(load().sv_hermitian_to_pauli(int(n), w.ctypes.data_as(_ip), k, m.view(np.float64).ctypes.data_as(_dp),
                                        float(tol), c.ctypes.data_as(_dp),
                                        x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                        z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(cnt)))
    out = []
    for t in range(cnt.value):
        letters = []
        for wire in range(n):
            xb, zb = (int(x[t]) >> wire) & 1, (int(z[t]) >> wire) & 1
            if xb or zb:
                letters.append((wire, "Y" if xb and zb else ("X" if xb else "Z")))
        out.append(PauliTerm(float(c[t]), tuple(letters)))
    return out


def sv_program_stats(ph: int):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().sv_program_stats(_vp(ph), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sv_plan_query(n: int, dtype: int, tape: "Tape"):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().sv_plan_query(int(n), int(dtype), ctypes.byref(tape.struct), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sv_kernel_timing_enable(enable: bool) -> None:
    _check(load().sv_kernel_timing_enable(int(bool(enable))))


def sv_kernel_timing_reset() -> None:
    _check(load().sv_kernel_timing_reset())


def sv_kernel_timing_read():
    """{class name: (total ms, launches)} of the launches bracketed so far."""
    ms = (ctypes.c_double * len(KERNEL_CLASSES))()
    cnt = (ctypes.c_int64 * len(KERNEL_CLASSES))()
    _check(load().sv_kernel_timing_read(ms, cnt))
    return {name: (ms[i], cnt[i]) for i, name in enumerate(KERNEL_CLASSES)}


class Batch:
    """Many circuits in one persistent, graph-captured launch (sv_batch_*).

    ``circuits``: objects with ``n``, ``ops``, ``n_params``, ``observables``
    (the first observable is measured; Z-only words) and ``basis_state``.
    Circuits that share a structure may pass the same object repeatedly.
    """

    def __init__(self, circuits, dtype: int = SV_C64):
        self.count = len(circuits)
        cache = {}
        tapes = (SvTape * self.count)()
        obs = []
        self._keep = []
        for i, c in enumerate(circuits):
            key = id(c)
            if key not in cache:
                cache[key] = Tape(c.ops, c.n_params)
            t = cache[key]
            self._keep.append(t)
            tapes[i] = t.struct
            obs.append(c.observables[0] if c.observables else [])
        self._tapes = tapes
        self._obs = PauliSums(obs)
        nq = (ctypes.c_int * self.count)(*[int(c.n) for c in circuits])
        basis = (ctypes.c_uint64 * self.count)(*[int(getattr(c, "basis_state", 0)) for c in circuits])
        self.n_params = sum(int(c.n_params) for c in circuits)
        h = _vp()
        _check(load().sv_batch_create(int(dtype), self.count, nq, tapes, self._obs.array, basis, ctypes.byref(h)))
        self.handle = h.value

    def set_params(self, params, on_device: bool = False) -> None:
        if on_device:
            _check(load().sv_batch_set_params(_vp(self.handle), _vp(params), 1))
        else:
            p = np.ascontiguousarray(params, dtype=np.float64).ravel()
            assert p.size == self.n_params
            _check(load().sv_batch_set_params(_vp(self.handle), p.ctypes.data_as(_vp), 0))

    def run(self) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.float64)
        _check(load().sv_batch_run(_vp(self.handle), out.ctypes.data_as(_vp), 0))
        return out

    def run_device(self, out_ptr: int) -> None:
        _check(load().sv_batch_run(_vp(self.handle), _vp(out_ptr), 1))

    def status(self) -> None:
        _check(load().sv_batch_status(_vp(self.handle)))

    def set_stream(self, stream: int) -> None:
        _check(load().sv_batch_set_stream(_vp(self.handle), _vp(stream)))

    def autotune(self) -> float:
        ms = ctypes.c_double()
        _check(load().sv_batch_autotune(_vp(self.handle), ctypes.byref(ms)))
        return ms.value

    def info(self):
        items, ctas, tbits, wave, graph = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        _check(load().sv_batch_info(_vp(self.handle), ctypes.byref(items), ctypes.byref(ctas), ctypes.byref(tbits),
                                    ctypes.byref(wave), ctypes.byref(graph)))
        return {"work_items": items.value, "ctas": ctas.value, "tile_bits": tbits.value,
                "wave_bytes": wave.value, "graph": bool(graph.value)}

    def close(self) -> None:
        if getattr(self, "handle", None):
            _check(load().sv_batch_destroy(_vp(self.handle)))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sv_expval_static(device_ptr: int, n: int, dtype: int, obs: "PauliSums", stream: int = 0) -> np.ndarray:
    """sv_expval for a state given by device pointer, with no device allocation
    (all temporaries in the library's fixed scratch array)."""
    out = np.zeros(obs.count, dtype=np.float64)
    _check(load().sv_expval_static(_vp(device_ptr), int(n), int(dtype), obs.array, obs.count, _dptr(out),
                                   _vp(stream)))
    return out


# ---------------------------------------------------------------------------
# Marshalling of circuits and observables into the C structs
# ---------------------------------------------------------------------------
class Tape:
    """An sv_tape built from a list of ops (objects with name / wires / params /
    controls / control_values / adjoint / scale, e.g. ``workloads.Op``)."""

    def __init__(self, ops, n_params: int, matrices: Optional[Sequence[np.ndarray]] = None):
        self.ops = (SvOp * max(1, len(ops)))()
        mats = []
        moff = 0
        for i, op in enumerate(ops):
            o = self.ops[i]
            o.kind = KIND[op.name]
            o.n_targets = len(op.wires)
            for j, w in enumerate(op.wires):
                o.targets[j] = int(w)
            ctrls = tuple(getattr(op, "controls", ()) or ())
            cvals = tuple(getattr(op, "control_values", ()) or ()) or (1,) * len(ctrls)
            o.n_controls = len(ctrls)
            for c, (w, v) in enumerate(zip(ctrls, cvals)):
                o.controls[c] = int(w)
                o.control_values[c] = int(v)
            pidx = tuple(getattr(op, "params", ()) or ())
            for a in range(3):
                o.param_index[a] = int(pidx[a]) if a < len(pidx) else -1
            consts = tuple(getattr(op, "constants", ()) or ())
            for a, v in enumerate(consts[:3]):
                o.const_angle[a] = float(v)
            o.scale = float(getattr(op, "scale", 1.0))
            o.adjoint = int(bool(getattr(op, "adjoint", False)))
            if op.name == "QubitUnitary":
                m = np.ascontiguousarray(op.matrix, dtype=np.complex128)
                o.matrix_offset = moff
                mats.append(m.ravel())
                moff += m.size
        self.matrices = (np.ascontiguousarray(np.concatenate(mats)).view(np.float64)
                         if mats else None)
        self.n_params = int(n_params)
        self.struct = SvTape(len(ops), self.ops, self.n_params, _dptr(self.matrices), moff)


class PauliSums:
    """A list of Hamiltonians (each a list of terms with ``coeff`` and
    ``paulis`` = ((wire, 'X'|'Y'|'Z'), ...)) as an sv_pauli_sum array."""

    def __init__(self, observables):
        self.count = len(observables)
        self.array = (SvPauliSum * max(1, self.count))()
        self._keep = []
        for j, H in enumerate(observables):
            c = np.array([float(t.coeff) for t in H], dtype=np.float64)
            x = np.zeros(len(H), dtype=np.uint64)
            z = np.zeros(len(H), dtype=np.uint64)
            for t, term in enumerate(H):
                xm = zm = 0
                for w, letter in term.paulis:
                    if letter in ("X", "Y"):
                        xm |= 1 << int(w)
                    if letter in ("Y", "Z"):
                        zm |= 1 << int(w)
                x[t], z[t] = xm, zm
            self._keep += [c, x, z]
            self.array[j] = SvPauliSum(len(H), c.ctypes.data_as(_dp),
                                       x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                       z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
