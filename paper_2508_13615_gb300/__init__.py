"""GB300 state-vector gate engine (arxiv 2508.13615's index-dependent,
gate-specific kernels, on one GPU).

The C ABI (``include/lqs.h``) is the product; :mod:`.lqs` binds it with the
same function names.  This module adds a thin convenience layer: a
``StateVector`` whose amplitudes live in a torch tensor, and an autograd
Function whose backward pass is the library's adjoint sweep.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import lqs
from .lqs import (BatchItems, GATE_IDS, LQS_ARITH_AUTO, LQS_ARITH_DF, LQS_ARITH_F64, LQS_C64, LQS_C128, LQS_JIT_AUTO, LQS_JIT_OFF,
                  LQS_JIT_ON, LqsError, OpArray,
                  PauliArray, lqs_adjoint_grad, lqs_apply_fused, lqs_apply_gate, lqs_apply_matrix, lqs_autotune_fused, lqs_batch_autotune, lqs_batch_run,
                  lqs_debug_df_roundtrip, lqs_expval, lqs_expval_static, lqs_jit_info, lqs_jit_precompile, lqs_jit_precompile_adjoint, lqs_jit_precompile_expval, lqs_kernel_launches, lqs_last_error, lqs_norm2,
                  lqs_plan_fused, lqs_profile_start, lqs_profile_stop, lqs_set_arith, lqs_set_jit, lqs_sv_alloc, lqs_sv_copy_from_host, lqs_sv_copy_to_host, lqs_sv_copy_to_host_async, lqs_apply_block, lqs_block_matrix, lqs_sv_distance,
                  lqs_sv_free, lqs_sv_info, lqs_sv_set_basis, lqs_sv_sync, lqs_version, lqs_check_bounded_wait)

__all__ = [n for n in dir(lqs) if n.startswith("lqs_")] + ["BatchItems", "StateVector", "ExpvalFunction",
                                                             "expval_autograd"]


class StateVector:
    """An n-qubit state in a CUDA torch tensor, with a library handle on it.

    The tensor (complex64 or complex128, 2^n entries) owns the memory; calls
    are ordered on the torch stream that was current at construction.
    """

    def __init__(self, n_qubits: int, dtype="c128", device: Optional[str] = None, tensor=None, stream=None):
        import torch
        self.n = int(n_qubits)
        code = lqs._dtype_code(dtype)
        tdt = torch.complex64 if code == LQS_C64 else torch.complex128
        if tensor is None:
            tensor = torch.empty(1 << self.n, dtype=tdt, device=device or "cuda")
        if tensor.dtype != tdt or tensor.numel() != (1 << self.n) or not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("tensor must be a contiguous CUDA tensor of 2^n amplitudes of the given dtype")
        self.tensor = tensor
        self.dtype = code
        self.stream = stream if stream is not None else torch.cuda.current_stream(tensor.device)
        self.h = lqs_sv_alloc(self.n, code, tensor.data_ptr(), self.stream.cuda_stream)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            lqs_sv_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- contents -----------------------------------------------------------
    def set_basis(self, x: int = 0) -> "StateVector":
        lqs_sv_set_basis(self.h, x)
        return self

    def from_numpy(self, a: np.ndarray) -> "StateVector":
        a = np.ascontiguousarray(a, dtype=np.complex64 if self.dtype == LQS_C64 else np.complex128)
        lqs_sv_copy_from_host(self.h, a)
        lqs_sv_sync(self.h)
        return self

    def numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == LQS_C64 else np.complex128)
        return lqs_sv_copy_to_host(self.h, out)

    def sync(self) -> None:
        lqs_sv_sync(self.h)

    # -- gates ----------------------------------------------------------------
    def apply_gate(self, name: str, wires: Sequence[int], params=(), inverse: bool = False) -> "StateVector":
        lqs_apply_gate(self.h, name, wires, params, inverse)
        return self

    def apply(self, circuit, fused: bool = True, cfg=None) -> "StateVector":
        """Apply a circuit (ops with .name .wires .pidx .matrix .inverse; .params)."""
        if fused:
            lqs_apply_fused(self.h, circuit.ops, circuit.params, cfg)
        else:
            for op in circuit.ops:
                k = lqs.GATE_NPARAMS.get(op.name, 0)
                if op.name in ("U2", "U4"):
                    p = op.matrix
                else:
                    p = circuit.params[op.pidx: op.pidx + k] if k else ()
                lqs_apply_gate(self.h, op.name, op.wires, p, op.inverse)
        return self

    # -- measurement ----------------------------------------------------------
    def norm2(self) -> float:
        return lqs_norm2(self.h)

    def expval(self, terms):
        return lqs_expval(self.h, terms)

    def adjoint_grad(self, circuit, terms):
        """(gradient, energy); the state must hold the circuit's output and is
        returned to the circuit's input state."""
        return lqs_adjoint_grad(self.h, circuit.ops, circuit.params, terms)


class ExpvalFunction:
    """torch.autograd.Function: E(params) = <0|U(params)^dag H U(params)|0>,
    forward on the fused path, backward by the library's adjoint sweep."""

    _fn = None

    @classmethod
    def get(cls):
        if cls._fn is None:
            import torch

            class _Expval(torch.autograd.Function):
                @staticmethod
                def forward(ctx, params, circuit, terms, dtype):
                    p = params.detach().to("cpu", torch.float64).numpy()
                    sv = StateVector(circuit.n_qubits, dtype)
                    sv.set_basis(0)
                    lqs_apply_fused(sv.h, circuit.ops, p, None)
                    e, _ = sv.expval(terms)
                    ctx.sv, ctx.circuit, ctx.terms, ctx.p = sv, circuit, terms, p
                    ctx.pdtype, ctx.pdevice = params.dtype, params.device
                    return torch.tensor(e, dtype=params.dtype, device=params.device)

                @staticmethod
                def backward(ctx, grad_out):
                    g, _ = lqs_adjoint_grad(ctx.sv.h, ctx.circuit.ops, ctx.p, ctx.terms)
                    ctx.sv.close()
                    gt = torch.as_tensor(g, dtype=ctx.pdtype, device=ctx.pdevice)
                    return gt * grad_out, None, None, None

            cls._fn = _Expval
        return cls._fn


def expval_autograd(params, circuit, terms, dtype="c128"):
    """Differentiable expectation value (see ExpvalFunction)."""
    return ExpvalFunction.get().apply(params, circuit, terms, dtype)
