"""PyTorch-facing objects over libsv.so.

PyTorch supplies device memory (the amplitude buffer and result tensors) and
the stream; every arithmetic step runs in the library's CUDA kernels.

* :class:`StateVector` -- a 2^n state in a torch tensor (complex64 / complex128).
* :class:`Program` -- a planned tape + observables: forward pass, expectation
  values, full adjoint Jacobian (the method of Sec. 2.2 / 4.3), VJP.
* :class:`AdjointExpval` -- ``torch.autograd.Function``: forward gives
  <H_j>(params), backward is one adjoint sweep with lambda = sum_j g_j H_j psi.
  The forward state psi stays in the program's state vector (the checkpoint),
  so a backward holds three vectors: psi, phi, lambda.
"""

from __future__ import annotations

import weakref
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

_DT = {"c64": (L.SV_C64, torch.complex64), "c128": (L.SV_C128, torch.complex128),
       "c128df": (L.SV_C128, torch.complex128),
       torch.complex64: (L.SV_C64, torch.complex64), torch.complex128: (L.SV_C128, torch.complex128)}


def _require_cuda(device) -> torch.device:
    dev = torch.device(device)
    if dev.type != "cuda":
        raise RuntimeError("the state-vector library runs on a CUDA device only (no CPU path)")
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: the state-vector library needs a GB300 GPU")
    return dev


class StateVector:
    """A 2^n-amplitude state held in a torch tensor on the GPU (wire 0 = MSB).

    dtype "c64" / "c128" (IEEE FP64 arithmetic) / "c128df" (complex128 storage,
    double-float arithmetic on the FP32 pipe).  renormalize: scale the state to
    unit norm (FP64 norm) after each circuit forward pass; None = the library
    default (on for c64, off for c128)."""

    def __init__(self, n: int, dtype="c128", device="cuda", basis_state: int = 0,
                 renormalize: Optional[bool] = None):
        dev = _require_cuda(device)
        self.n = int(n)
        self.sv_dtype, self.torch_dtype = _DT[dtype]
        with torch.cuda.device(dev):
            self.tensor = torch.empty(1 << self.n, dtype=self.torch_dtype, device=dev)
            self.handle = L.sv_create_from_device_ptr(self.n, self.sv_dtype, self.tensor.data_ptr())
        self.device = dev
        self.generation = 0
        self._programs = weakref.WeakSet()  # programs on this state: closed before it
        if dtype == "c128df":
            L.sv_set_compute(self.handle, L.SV_COMPUTE_DOUBLE_FLOAT)
        if renormalize is not None:
            L.sv_set_renormalize(self.handle, bool(renormalize))
        self.sync_stream()
        self.reset(basis_state)

    def sync_stream(self) -> None:
        L.sv_set_stream(self.handle, torch.cuda.current_stream(self.device).cuda_stream)

    def reset(self, basis_state: int = 0) -> "StateVector":
        L.sv_reset(self.handle, int(basis_state))
        self.generation += 1
        return self

    def apply(self, name: str, wires: Sequence[int], angles: Sequence[float] = (), adjoint: bool = False):
        L.sv_apply(self.handle, L.KIND[name], list(wires), list(angles), adjoint)
        self.generation += 1
        return self

    def apply_matrix(self, wires: Sequence[int], matrix, adjoint: bool = False):
        L.sv_apply_matrix(self.handle, list(wires), np.asarray(matrix), adjoint)
        self.generation += 1
        return self

    def expval(self, observables) -> np.ndarray:
        return L.sv_expval(self.handle, L.PauliSums(observables))

    def var(self, observables) -> np.ndarray:
        return L.sv_var(self.handle, L.PauliSums(observables))

    def probs(self, wires) -> np.ndarray:
        return L.sv_probs(self.handle, list(wires))

    def sample(self, wires, uniforms) -> np.ndarray:
        return L.sv_sample(self.handle, list(wires), uniforms)

    def norm2(self) -> float:
        return L.sv_norm2(self.handle)

    def to_numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.sv_dtype == L.SV_C64 else np.complex128)
        return L.sv_get_state(self.handle, out)

    def set_numpy(self, amps: np.ndarray) -> None:
        a = np.ascontiguousarray(amps, dtype=np.complex64 if self.sv_dtype == L.SV_C64 else np.complex128)
        L.sv_set_state(self.handle, a)
        self.generation += 1

    def close(self) -> None:
        if getattr(self, "handle", None):
            for prog in list(getattr(self, "_programs", ())):
                prog.close()  # a program refers to its state's handle
            L.sv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Program:
    """A tape (ops over ``n_params`` parameters) and observables planned once."""

    def __init__(self, sv: StateVector, ops, n_params: int, observables=None, basis_state: int = 0):
        self.sv = sv
        self.tape = L.Tape(ops, n_params)
        self.obs = L.PauliSums(observables) if observables else None
        self.m = self.obs.count if self.obs else 0
        self.n_params = int(n_params)
        self.basis_state = int(basis_state)
        if not getattr(sv, "handle", None):
            raise RuntimeError("the state vector is closed")
        self.handle = L.sv_program_create(sv.handle, self.tape, self.obs)
        sv._programs.add(self)
        self._params = torch.zeros(max(1, self.n_params), dtype=torch.float64, device=sv.device)
        self._forward_generation = None

    @classmethod
    def from_circuit(cls, sv: StateVector, circuit, observables=None):
        obs = circuit.observables if observables is None else observables
        return cls(sv, circuit.ops, circuit.n_params, obs, circuit.basis_state)

    def set_params(self, params) -> None:
        if not torch.is_tensor(params):
            params = torch.as_tensor(np.asarray(params, dtype=np.float64))
        p = params.detach().to(device=self.sv.device, dtype=torch.float64).contiguous()
        if p.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.numel()}")
        if self.n_params:
            self._params[: self.n_params].copy_(p)
        self.sv.sync_stream()
        L.sv_program_set_params(self.handle, self._params.data_ptr(), True)

    def forward(self, params=None, reset: bool = True) -> None:
        """psi = U(params)|basis_state>  (from the current state if reset=False)."""
        if params is not None:
            self.set_params(params)
        self.sv.sync_stream()
        if reset:
            self.sv.reset(self.basis_state)
        L.sv_program_forward(self.handle)
        self.sv.generation += 1
        self._forward_generation = self.sv.generation

    def expval(self) -> torch.Tensor:
        out = torch.empty(self.m, dtype=torch.float64, device=self.sv.device)
        self.sv.sync_stream()
        L.sv_program_expval(self.handle, out.data_ptr(), True)
        return out

    def jacobian(self):
        """(E, J) as device tensors: E[j] = <H_j>, J[j, p] = dE_j / dparams[p]."""
        E = torch.empty(self.m, dtype=torch.float64, device=self.sv.device)
        J = torch.empty((self.m, self.n_params), dtype=torch.float64, device=self.sv.device)
        self.sv.sync_stream()
        L.sv_program_jacobian(self.handle, E.data_ptr(), J.data_ptr(), True)
        return E, J

    def vjp(self, grad_out) -> torch.Tensor:
        g = np.ascontiguousarray(torch.as_tensor(grad_out).detach().double().cpu().numpy().ravel())
        out = torch.empty(max(1, self.n_params), dtype=torch.float64, device=self.sv.device)
        self.sv.sync_stream()
        L.sv_program_vjp(self.handle, g, out.data_ptr(), True)
        return out[: self.n_params]

    def jvp(self, tangent, reset: bool = True) -> torch.Tensor:
        """Forward-mode J @ tangent (one tangent pass from the basis state, or from
        the current state if reset=False); the state ends as the forward output."""
        t = np.ascontiguousarray(torch.as_tensor(tangent).detach().double().cpu().numpy().ravel())
        if t.size != self.n_params:
            raise ValueError(f"expected {self.n_params} tangent entries, got {t.size}")
        out = torch.empty(max(1, self.m), dtype=torch.float64, device=self.sv.device)
        self.sv.sync_stream()
        if reset:
            self.sv.reset(self.basis_state)
        L.sv_program_jvp(self.handle, t, out.data_ptr(), True)
        self.sv.generation += 1
        self._forward_generation = self.sv.generation
        return out[: self.m]

    def jacobian_by_shape(self):
        """(E, J) by whichever mode costs fewer passes: reverse mode (one adjoint
        sweep per observable, `jacobian`) unless there are fewer parameters than
        observables, then forward mode (one tangent pass per parameter)."""
        if self.n_params >= self.m:
            self.forward()
            return self.jacobian()
        J = torch.empty((self.m, self.n_params), dtype=torch.float64, device=self.sv.device)
        eye = np.eye(self.n_params)
        for q in range(self.n_params):
            J[:, q] = self.jvp(eye[q])
        return self.expval(), J

    def stats(self):
        return L.sv_program_stats(self.handle)

    def state_is_forward_output(self) -> bool:
        return self._forward_generation == self.sv.generation

    def close(self) -> None:
        if getattr(self, "handle", None):
            L.sv_program_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdjointExpval(torch.autograd.Function):
    """E = <psi(params)|H_j|psi(params)>; backward = adjoint VJP on the GPU."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, program: Program):
        program.forward(params)
        ctx.program = program
        ctx.generation = program.sv.generation
        ctx.param_device = params.device
        return program.expval().to(params.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        program: Program = ctx.program
        if program.sv.generation != ctx.generation:
            raise RuntimeError("the state vector changed between forward and backward; "
                               "run backward before reusing the program")
        g = program.vjp(grad_out)
        return g.to(ctx.param_device), None


def expval(params: torch.Tensor, program: Program) -> torch.Tensor:
    """Differentiable expectation values of the program's observables."""
    return AdjointExpval.apply(params, program)
