"""ctypes binding of the C ABI in ``include/lqs.h`` (same function names).

Argument marshalling only: every step of gate application, measurement and
differentiation runs in the CUDA library.  PyTorch supplies device memory and
streams.  If the library has not been built this module raises ImportError;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblqs.so")

LQS_OK = 0
LQS_ERR_ARG = -1
LQS_ERR_OOM = -2
LQS_ERR_CUDA = -3
LQS_ERR_TIMEOUT = -4
LQS_ERR_UNSUPPORTED = -5
LQS_C64 = 0
LQS_C128 = 1
LQS_ARITH_AUTO, LQS_ARITH_F64, LQS_ARITH_DF = 0, 1, 2
LQS_JIT_OFF, LQS_JIT_ON, LQS_JIT_AUTO = 0, 1, 2

#: gate ids of the ABI (lqs_gate), by the names used in circuit descriptions
GATE_IDS = {
    "X": 0, "Y": 1, "Z": 2, "H": 3, "S": 4, "T": 5, "RX": 6, "RY": 7, "RZ": 8, "PhaseShift": 9, "Rot": 10,
    "CNOT": 11, "CZ": 12, "SWAP": 13, "ControlledPhaseShift": 14, "CRY": 15, "Toffoli": 16, "U2": 17, "U4": 18,
    "CSWAP": 19, "DoubleExcitation": 20,
}
GATE_NWIRES = {"X": 1, "Y": 1, "Z": 1, "H": 1, "S": 1, "T": 1, "RX": 1, "RY": 1, "RZ": 1, "PhaseShift": 1, "Rot": 1,
               "CNOT": 2, "CZ": 2, "SWAP": 2, "ControlledPhaseShift": 2, "CRY": 2, "Toffoli": 3, "U2": 1, "U4": 2,
               "CSWAP": 3, "DoubleExcitation": 4}
GATE_NPARAMS = {"RX": 1, "RY": 1, "RZ": 1, "PhaseShift": 1, "Rot": 3, "ControlledPhaseShift": 1, "CRY": 1,
                "DoubleExcitation": 1}


class lqs_op(ctypes.Structure):
    _fields_ = [("gate", ctypes.c_int32), ("wires", ctypes.c_int32 * 4), ("param_idx", ctypes.c_int32),
                ("inverse", ctypes.c_int32), ("matrix", ctypes.POINTER(ctypes.c_double))]


class lqs_pauli(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64)]


class lqs_fuse_cfg(ctypes.Structure):
    _fields_ = [("tile_qubits", ctypes.c_int32), ("low_qubits", ctypes.c_int32), ("arith", ctypes.c_int32),
                ("max_ops", ctypes.c_int32), ("tc_blocks", ctypes.c_int32)]


class lqs_batch_item(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_ops", ctypes.c_int32), ("ops", ctypes.POINTER(lqs_op)),
                ("n_params", ctypes.c_int32), ("params", ctypes.POINTER(ctypes.c_double)),
                ("n_terms", ctypes.c_int32), ("terms", ctypes.POINTER(lqs_pauli)),
                ("grads", ctypes.POINTER(ctypes.c_double)), ("energy", ctypes.POINTER(ctypes.c_double))]


class lqs_launch_record(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 48), ("ms", ctypes.c_float), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double)]


class lqs_jit_stats(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("compiled", ctypes.c_int), ("failed", ctypes.c_int),
                ("cached", ctypes.c_int), ("launches", ctypes.c_uint64), ("compile_seconds", ctypes.c_double),
                ("last_error", ctypes.c_char * 256)]


class LqsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lqs error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    i32, u64, i64 = ctypes.c_int, ctypes.c_uint64, ctypes.c_int64
    sig = {
        "lqs_sv_alloc": (i32, [i32, i32, vp, vp, ctypes.POINTER(vp)]),
        "lqs_sv_free": (i32, [vp]),
        "lqs_sv_info": (i32, [vp, ctypes.POINTER(vp), ip, ip]),
        "lqs_sv_set_basis": (i32, [vp, u64]),
        "lqs_sv_copy_from_host": (i32, [vp, vp]),
        "lqs_sv_copy_to_host": (i32, [vp, vp]),
        "lqs_sv_copy_to_host_async": (i32, [vp, vp]),
        "lqs_apply_block": (i32, [vp, ctypes.c_int, vp]),
        "lqs_block_matrix": (i32, [vp, ctypes.c_int, vp, ctypes.c_int, vp]),
        "lqs_sv_sync": (i32, [vp]),
        "lqs_check_bounded_wait": (i32, [vp]),
        "lqs_apply_gate": (i32, [vp, i32, ip, i32, dp, i32, i32]),
        "lqs_apply_matrix": (i32, [vp, ip, i32, dp]),
        "lqs_apply_fused": (i32, [vp, ctypes.POINTER(lqs_op), i32, dp, i32, ctypes.POINTER(lqs_fuse_cfg)]),
        "lqs_plan_fused": (i32, [i32, i32, ctypes.POINTER(lqs_op), i32, ctypes.POINTER(lqs_fuse_cfg), ip,
                                 ctypes.POINTER(u64), i32, ip]),
        "lqs_norm2": (i32, [vp, dp]),
        "lqs_expval": (i32, [vp, ctypes.POINTER(lqs_pauli), i32, dp, dp]),
        "lqs_adjoint_grad": (i32, [vp, ctypes.POINTER(lqs_op), i32, dp, i32, ctypes.POINTER(lqs_pauli), i32, dp,
                                   dp]),
        "lqs_batch_run": (i32, [ctypes.POINTER(lqs_batch_item), i32, i32, vp]),
        "lqs_batch_autotune": (i32, [ctypes.POINTER(lqs_batch_item), i32, i32, vp, i32, ip]),
        "lqs_last_error": (ctypes.c_char_p, []),
        "lqs_version": (i32, []),
        "lqs_set_arith": (i32, [i32]),
        "lqs_kernel_launches": (u64, []),
        "lqs_debug_df_roundtrip": (i32, [dp, dp, i64]),
        "lqs_expval_static": (i32, [vp, i32, i32, vp, ctypes.POINTER(lqs_pauli), i32, dp, dp]),
        "lqs_sv_distance": (i32, [vp, vp, dp, dp]),
        "lqs_profile_start": (i32, []),
        "lqs_profile_stop": (i32, [ctypes.POINTER(lqs_launch_record), i32, ip]),
        "lqs_set_jit": (i32, [i32]),
        "lqs_jit_info": (i32, [ctypes.POINTER(lqs_jit_stats)]),
        "lqs_jit_precompile": (i32, [i32, i32, i32, ctypes.POINTER(lqs_op), i32, dp, i32,
                                     ctypes.POINTER(lqs_fuse_cfg), ip]),
        "lqs_jit_precompile_adjoint": (i32, [i32, i32, i32, ctypes.POINTER(lqs_op), i32, dp, i32, ip]),
        "lqs_jit_precompile_expval": (i32, [i32, i32, i32, ctypes.POINTER(lqs_pauli), i32, i32, ip]),
        "lqs_autotune_fused": (i32, [vp, ctypes.POINTER(lqs_op), i32, dp, i32, i32, ctypes.POINTER(lqs_fuse_cfg)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_L = _load()


def _check(rc: int) -> int:
    if rc != LQS_OK:
        raise LqsError(rc, _L.lqs_last_error().decode(errors="replace"))
    return rc


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dtype_code(dtype) -> int:
    if dtype in (LQS_C64, "c64", "complex64", np.complex64):
        return LQS_C64
    if dtype in (LQS_C128, "c128", "complex128", np.complex128):
        return LQS_C128
    try:
        import torch
        if dtype == torch.complex64:
            return LQS_C64
        if dtype == torch.complex128:
            return LQS_C128
    except ImportError:
        pass
    raise ValueError(f"unknown dtype {dtype!r}")


# ---------------------------------------------------------------------------
# marshalling of circuits and observables
# ---------------------------------------------------------------------------

class OpArray:
    """ctypes array of lqs_op built from ops with .name .wires .pidx .matrix .inverse."""

    def __init__(self, ops: Sequence):
        self.n = len(ops)
        self.arr = (lqs_op * max(self.n, 1))()
        self._mats: List[np.ndarray] = []
        for i, op in enumerate(ops):
            rec = self.arr[i]
            rec.gate = GATE_IDS[op.name]
            w = list(op.wires)
            for j in range(4):
                rec.wires[j] = int(w[j]) if j < len(w) else 0
            rec.param_idx = int(op.pidx) if getattr(op, "pidx", -1) is not None else -1
            rec.inverse = int(bool(getattr(op, "inverse", False)))
            m = getattr(op, "matrix", None)
            if m is not None:
                mm = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(-1)).view(np.float64).copy()
                self._mats.append(mm)
                rec.matrix = _dptr(mm)
            else:
                rec.matrix = None

    def ptr(self):
        return ctypes.cast(self.arr, ctypes.POINTER(lqs_op))


class PauliArray:
    def __init__(self, terms: Iterable):
        terms = list(terms)
        self.n = len(terms)
        self.arr = (lqs_pauli * max(self.n, 1))()
        for i, t in enumerate(terms):
            self.arr[i].coeff = float(t.coeff)
            self.arr[i].x_mask = int(t.x_mask)
            self.arr[i].z_mask = int(t.z_mask)

    def ptr(self):
        return ctypes.cast(self.arr, ctypes.POINTER(lqs_pauli))


def _cfg(cfg) -> Optional[lqs_fuse_cfg]:
    if cfg is None:
        return None
    if isinstance(cfg, lqs_fuse_cfg):
        return cfg
    c = lqs_fuse_cfg()
    c.tile_qubits = int(cfg.get("tile_qubits", 0))
    c.low_qubits = int(cfg.get("low_qubits", 0))
    c.arith = int(cfg.get("arith", 0))
    c.max_ops = int(cfg.get("max_ops", 0))
    c.tc_blocks = int(cfg.get("tc_blocks", 0))
    return c


def _params(params) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(params if params is not None else [], dtype=np.float64).reshape(-1))
    return p if p.size else np.zeros(1)


# ---------------------------------------------------------------------------
# the ABI, one Python function per C function
# ---------------------------------------------------------------------------

def lqs_sv_alloc(n_qubits: int, dtype, device_ptr: Optional[int] = None, cuda_stream: Optional[int] = None):
    h = ctypes.c_void_p()
    _check(_L.lqs_sv_alloc(int(n_qubits), _dtype_code(dtype), device_ptr, cuda_stream, ctypes.byref(h)))
    return h


def lqs_sv_free(h) -> None:
    _check(_L.lqs_sv_free(h))


def lqs_sv_info(h) -> Tuple[int, int, int]:
    p, n, d = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int()
    _check(_L.lqs_sv_info(h, ctypes.byref(p), ctypes.byref(n), ctypes.byref(d)))
    return p.value, n.value, d.value


def lqs_sv_set_basis(h, x: int) -> None:
    _check(_L.lqs_sv_set_basis(h, int(x)))


def lqs_sv_copy_from_host(h, host: np.ndarray) -> None:
    if not host.flags.c_contiguous:
        raise ValueError("host buffer must be contiguous")
    _check(_L.lqs_sv_copy_from_host(h, host.ctypes.data))


def lqs_sv_copy_to_host(h, host: np.ndarray) -> np.ndarray:
    if not host.flags.c_contiguous:
        raise ValueError("host buffer must be contiguous")
    _check(_L.lqs_sv_copy_to_host(h, host.ctypes.data))
    return host


def lqs_sv_copy_to_host_async(h, host: np.ndarray) -> np.ndarray:
    """Enqueues the copy only; ``host`` holds the state after lqs_sv_sync(h)."""
    if not host.flags.c_contiguous:
        raise ValueError("host buffer must be contiguous")
    _check(_L.lqs_sv_copy_to_host_async(h, host.ctypes.data))
    return host


def lqs_apply_block(h, m: int, matrix) -> None:
    """Dense 2^m x 2^m complex matrix on qubits 0..m-1 (tensor cores; complex64, m = 5)."""
    U = np.ascontiguousarray(matrix, dtype=np.complex128)
    if U.shape != (1 << m, 1 << m):
        raise ValueError("matrix must be 2^m x 2^m")
    _check(_L.lqs_apply_block(h, int(m), U.ctypes.data))


def lqs_block_matrix(ops, params) -> np.ndarray:
    """The 32x32 complex matrix of a run of gates on qubits 0..4 (host only)."""
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    p = _params(params)
    out = np.zeros((32, 32), dtype=np.complex128)
    _check(_L.lqs_block_matrix(oa.ptr(), oa.n, _dptr(p), int(np.asarray(params).size) if params is not None else 0,
                               out.ctypes.data))
    return out


def lqs_sv_sync(h) -> None:
    _check(_L.lqs_sv_sync(h))


def lqs_check_bounded_wait(h) -> None:
    """Enqueues a kernel whose bounded wait gives up; the next lqs_sv_sync(h) raises LQS_ERR_TIMEOUT."""
    _check(_L.lqs_check_bounded_wait(h))


def lqs_apply_gate(h, gate, wires: Sequence[int], params=(), inverse: bool = False) -> None:
    """One gate on the plain path; U2/U4 take their matrix as ``params``."""
    gid = GATE_IDS[gate] if isinstance(gate, str) else int(gate)
    w = (ctypes.c_int * max(len(wires), 1))(*[int(x) for x in wires])
    if gid in (GATE_IDS["U2"], GATE_IDS["U4"]):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.complex128).reshape(-1)).view(np.float64).copy()
        npar = int(p.size)
    else:
        npar = int(np.asarray(params, dtype=np.float64).size)
        p = _params(params)
    _check(_L.lqs_apply_gate(h, gid, w, len(wires), _dptr(p), npar, int(bool(inverse))))


def lqs_apply_matrix(h, wires: Sequence[int], matrix) -> None:
    w = (ctypes.c_int * max(len(wires), 1))(*[int(x) for x in wires])
    m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128).reshape(-1)).view(np.float64).copy()
    _check(_L.lqs_apply_matrix(h, w, len(wires), _dptr(m)))


def lqs_apply_fused(h, ops, params, cfg=None) -> None:
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    p = _params(params)
    c = _cfg(cfg)
    _check(_L.lqs_apply_fused(h, oa.ptr(), oa.n, _dptr(p), int(np.asarray(params).size) if params is not None else 0,
                              ctypes.byref(c) if c is not None else None))


def lqs_plan_fused(n_qubits: int, dtype, ops, cfg=None):
    """(n_segments, segment qubit masks, segment of each op) -- host only."""
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    c = _cfg(cfg)
    nseg = ctypes.c_int()
    cap = max(oa.n, 1)
    masks = (ctypes.c_uint64 * cap)()
    seg_of = (ctypes.c_int * cap)()
    _check(_L.lqs_plan_fused(int(n_qubits), _dtype_code(dtype), oa.ptr(), oa.n,
                             ctypes.byref(c) if c is not None else None, ctypes.byref(nseg), masks, cap, seg_of))
    return nseg.value, [int(masks[i]) for i in range(min(nseg.value, cap))], [int(seg_of[i]) for i in range(oa.n)]


def lqs_norm2(h) -> float:
    out = ctypes.c_double()
    _check(_L.lqs_norm2(h, ctypes.byref(out)))
    return out.value


def lqs_expval(h, terms) -> Tuple[float, np.ndarray]:
    pa = terms if isinstance(terms, PauliArray) else PauliArray(terms)
    out = ctypes.c_double()
    per = np.zeros(max(pa.n, 1), dtype=np.float64)
    _check(_L.lqs_expval(h, pa.ptr(), pa.n, ctypes.byref(out), _dptr(per)))
    return out.value, per[: pa.n]


def lqs_adjoint_grad(h, ops, params, terms) -> Tuple[np.ndarray, float]:
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    pa = terms if isinstance(terms, PauliArray) else PauliArray(terms)
    npar = int(np.asarray(params).size) if params is not None else 0
    p = _params(params)
    g = np.zeros(max(npar, 1), dtype=np.float64)
    e = ctypes.c_double()
    _check(_L.lqs_adjoint_grad(h, oa.ptr(), oa.n, _dptr(p), npar, pa.ptr(), pa.n, _dptr(g), ctypes.byref(e)))
    return g[:npar], e.value


def _batch_items(circuits: Sequence, terms_per_circuit: Sequence, grads: bool):
    m = len(circuits)
    items = (lqs_batch_item * max(m, 1))()
    keep = []
    energies = np.zeros(max(m, 1), dtype=np.float64)
    gl = []
    for i, (c, t) in enumerate(zip(circuits, terms_per_circuit)):
        oa = OpArray(c.ops)
        pa = PauliArray(t)
        p = _params(c.params)
        g = np.zeros(max(len(c.params), 1), dtype=np.float64)
        keep += [oa, pa, p, g]
        gl.append(g[: len(c.params)])
        it = items[i]
        it.n_qubits = c.n_qubits
        it.n_ops = oa.n
        it.ops = oa.ptr()
        it.n_params = len(c.params)
        it.params = _dptr(p)
        it.n_terms = pa.n
        it.terms = pa.ptr()
        it.grads = _dptr(g) if grads else None
        it.energy = ctypes.cast(ctypes.c_void_p(energies.ctypes.data + 8 * i), ctypes.POINTER(ctypes.c_double))
    return items, keep, energies, gl


class BatchItems:
    """The lqs_batch_item array of a batch, marshalled once.  `params[i]` is
    circuit i's parameter array as the library reads it: a variational loop
    writes new values into it in place and calls run() again."""

    def __init__(self, circuits: Sequence, terms_per_circuit: Sequence, grads: bool = True):
        self.m = len(circuits)
        self.items, self._keep, self._energies, self._grads = _batch_items(circuits, terms_per_circuit, grads)
        self.params = [self._keep[4 * i + 2] for i in range(self.m)]

    def run(self, dtype, cuda_stream: Optional[int] = None):
        """lqs_batch_run on the marshalled items; returns (energies, [grads]) (views, overwritten by the next run)."""
        _check(_L.lqs_batch_run(self.items, self.m, _dtype_code(dtype), cuda_stream))
        return self._energies[: self.m], self._grads

    def autotune(self, dtype, cuda_stream: Optional[int] = None, repeats: int = 2) -> int:
        n = ctypes.c_int()
        _check(_L.lqs_batch_autotune(self.items, self.m, _dtype_code(dtype), cuda_stream, int(repeats),
                                     ctypes.byref(n)))
        return n.value


def lqs_batch_run(circuits: Sequence, terms_per_circuit: Sequence, dtype, cuda_stream: Optional[int] = None,
                  grads: bool = True):
    """Forward + energy (+ adjoint gradients) of many circuits; returns (energies, [grads])."""
    m = len(circuits)
    items, keep, energies, gl = _batch_items(circuits, terms_per_circuit, grads)
    _check(_L.lqs_batch_run(items, m, _dtype_code(dtype), cuda_stream))
    return energies[:m], gl


def lqs_batch_autotune(circuits: Sequence, terms_per_circuit: Sequence, dtype, cuda_stream: Optional[int] = None,
                       repeats: int = 2, grads: bool = True) -> int:
    """Times the batch kernel's tile shapes per qubit count and keeps the fastest; returns how many counts were tuned."""
    m = len(circuits)
    items, keep, energies, gl = _batch_items(circuits, terms_per_circuit, grads)
    n = ctypes.c_int()
    _check(_L.lqs_batch_autotune(items, m, _dtype_code(dtype), cuda_stream, int(repeats), ctypes.byref(n)))
    return n.value


def lqs_last_error() -> str:
    return _L.lqs_last_error().decode(errors="replace")


def lqs_version() -> int:
    return int(_L.lqs_version())


def lqs_set_arith(arith: int) -> None:
    _check(_L.lqs_set_arith(int(arith)))


def lqs_kernel_launches() -> int:
    return int(_L.lqs_kernel_launches())


def lqs_debug_df_roundtrip(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2 * x.size, dtype=np.float64)
    _check(_L.lqs_debug_df_roundtrip(_dptr(x), _dptr(out), x.size))
    return out.reshape(-1, 2)


def lqs_profile_start() -> None:
    _check(_L.lqs_profile_start())


def lqs_profile_stop():
    """Per-launch records since lqs_profile_start: list of (kernel, ms, bytes, flops)."""
    cnt = ctypes.c_int()
    _check(_L.lqs_profile_stop(None, 0, ctypes.byref(cnt)))
    # the records stay until the next start: fetch them all
    recs = (lqs_launch_record * max(cnt.value, 1))()
    _check(_L.lqs_profile_stop(recs, cnt.value, ctypes.byref(cnt)))
    return [(r.kernel.decode(), float(r.ms), float(r.bytes), float(r.flops)) for r in recs[: cnt.value]]


def lqs_expval_static(psi_device_ptr: int, n_qubits: int, dtype, terms, cuda_stream: Optional[int] = None):
    """Allocation-free <psi|H|psi> over a raw device pointer (see include/lqs.h)."""
    pa = terms if isinstance(terms, PauliArray) else PauliArray(terms)
    out = ctypes.c_double()
    per = np.zeros(max(pa.n, 1), dtype=np.float64)
    _check(_L.lqs_expval_static(ctypes.c_void_p(psi_device_ptr), int(n_qubits), _dtype_code(dtype), cuda_stream,
                                pa.ptr(), pa.n, ctypes.byref(out), _dptr(per)))
    return out.value, per[: pa.n]


def lqs_sv_distance(ha, hb) -> Tuple[float, float]:
    """(sum |a-b|^2, sum |b|^2) in float64."""
    d, nb = ctypes.c_double(), ctypes.c_double()
    _check(_L.lqs_sv_distance(ha, hb, ctypes.byref(d), ctypes.byref(nb)))
    return d.value, nb.value


def lqs_set_jit(mode: int) -> None:
    """Segment-compiler mode: LQS_JIT_OFF, LQS_JIT_ON or LQS_JIT_AUTO."""
    _check(_L.lqs_set_jit(int(mode)))


def lqs_jit_info() -> dict:
    st = lqs_jit_stats()
    _check(_L.lqs_jit_info(ctypes.byref(st)))
    return {"mode": st.mode, "compiled": st.compiled, "failed": st.failed, "cached": st.cached,
            "launches": int(st.launches), "compile_seconds": float(st.compile_seconds),
            "last_error": st.last_error.decode(errors="replace")}


def lqs_jit_precompile(n_qubits: int, dtype, ops, params=None, arith: int = LQS_ARITH_AUTO, cfg=None) -> int:
    """Compiles (host only) the segment kernels lqs_apply_fused would launch; returns how many."""
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    p = _params(params)
    c = _cfg(cfg)
    n = ctypes.c_int()
    _check(_L.lqs_jit_precompile(int(n_qubits), _dtype_code(dtype), int(arith), oa.ptr(), oa.n, _dptr(p),
                                 int(np.asarray(params).size) if params is not None else 0,
                                 ctypes.byref(c) if c is not None else None, ctypes.byref(n)))
    return n.value


def lqs_jit_precompile_adjoint(n_qubits: int, dtype, ops, params=None, arith: int = LQS_ARITH_AUTO) -> int:
    """Compiles (host only) the reverse-sweep kernels lqs_adjoint_grad would launch; returns how many."""
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    p = _params(params)
    n = ctypes.c_int()
    _check(_L.lqs_jit_precompile_adjoint(int(n_qubits), _dtype_code(dtype), int(arith), oa.ptr(), oa.n, _dptr(p),
                                         int(np.asarray(params).size) if params is not None else 0, ctypes.byref(n)))
    return n.value


def lqs_jit_precompile_expval(n_qubits: int, dtype, terms, lambda_: bool = False, arith: int = LQS_ARITH_AUTO) -> int:
    """Compiles (host only) the Pauli-pass kernels of lqs_expval (or, with lambda_, of the adjoint's
    lambda = H psi); returns how many."""
    pa = terms if isinstance(terms, PauliArray) else PauliArray(terms)
    n = ctypes.c_int()
    _check(_L.lqs_jit_precompile_expval(int(n_qubits), _dtype_code(dtype), int(arith), pa.ptr(), pa.n,
                                        1 if lambda_ else 0, ctypes.byref(n)))
    return n.value


def lqs_autotune_fused(h, ops, params, repeats: int = 2) -> dict:
    """Times fused-path configurations on this state (used as scratch); returns the fastest, which later
    lqs_apply_fused calls without a cfg use for this circuit structure."""
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    p = _params(params)
    best = lqs_fuse_cfg()
    _check(_L.lqs_autotune_fused(h, oa.ptr(), oa.n, _dptr(p), int(np.asarray(params).size) if params is not None else 0,
                                 int(repeats), ctypes.byref(best)))
    return {"tile_qubits": best.tile_qubits, "low_qubits": best.low_qubits, "arith": best.arith,
            "max_ops": best.max_ops}
