"""CPU oracle of the state-vector gate engine -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA path: it applies
every gate as its full unitary matrix to index groups (the "general approach"
of Sec. 3.1 of arxiv 2508.13615) in plain C complex128 (``lqs_oracle.c``), and
this module only marshals arguments and sequences calls.

Parity status per function (what pins each, see ``tests/test_oracle_pins.py``):
  gate_matrix / op_matrix / apply_matrix / apply_op / run_circuit
      -- Kronecker-product brute force, matrix exponentials of the Pauli
      generators, gate identities, GHZ and QFT closed forms, numpy FFT.
  norm2 / expval / energy  -- explicit Kronecker Pauli matrices, eigenstates
      with known eigenvalues.
  param_shift_grad  -- central finite differences and the analytic derivative
      of closed-form one-qubit expectations.
  apply_matrix_at / apply_op_at  -- the full update at the same indices.
"""
from __future__ import annotations

import ctypes
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from workloads import GATE_ID, GATE_NPARAMS, GATE_WIRES, Circuit, Op, Pauli

from .build import LIB, build

_lib = None


def lib():
    """Loads (building first if needed) the oracle's shared library."""
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_uint64)
        L.oracle_gate_matrix.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, ip]
        L.oracle_gate_matrix.restype = ctypes.c_int
        L.oracle_apply_matrix.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp]
        L.oracle_apply_matrix.restype = None
        L.oracle_apply_matrix_at.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp, up, ctypes.c_int64, dp]
        L.oracle_apply_matrix_at.restype = None
        L.oracle_apply_gate.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp, dp, ctypes.c_int]
        L.oracle_apply_gate.restype = ctypes.c_int
        L.oracle_run.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp, dp]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_norm2.argtypes = [dp, ctypes.c_int]
        L.oracle_norm2.restype = ctypes.c_double
        L.oracle_pauli_expval.argtypes = [dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_pauli_expval.restype = ctypes.c_double
        L.oracle_expval.argtypes = [dp, ctypes.c_int, dp, up, up, ctypes.c_int, dp]
        L.oracle_expval.restype = ctypes.c_double
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _up(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _check_state(psi: np.ndarray, n: int) -> None:
    if psi.dtype != np.complex128 or psi.shape != (1 << n,) or not psi.flags.c_contiguous:
        raise ValueError("oracle states are contiguous complex128 vectors of length 2^n")


def gate_matrix(name: str, params: Sequence[float] = (), matrix: Optional[np.ndarray] = None,
                inverse: bool = False) -> np.ndarray:
    """The gate's 2^m x 2^m unitary (first listed wire = most significant bit)."""
    p = np.zeros(4, dtype=np.float64)
    p[: len(params)] = np.asarray(params, dtype=np.float64)
    user = np.zeros(32, dtype=np.float64)
    if matrix is not None:
        m = np.ascontiguousarray(matrix, dtype=np.complex128).reshape(-1)
        user[: 2 * m.size] = m.view(np.float64)
    out = np.zeros(512, dtype=np.float64)
    mm = ctypes.c_int(0)
    if lib().oracle_gate_matrix(GATE_ID[name], _dp(p), _dp(user), int(inverse), _dp(out), ctypes.byref(mm)):
        raise ValueError(name)
    d = 1 << mm.value
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def apply_matrix(psi: np.ndarray, n: int, wires: Sequence[int], U: np.ndarray) -> np.ndarray:
    """In place: psi <- U_full psi for U on ``wires``."""
    _check_state(psi, n)
    w = np.asarray(wires, dtype=np.int32)
    if not 1 <= len(w) <= 7 or U.shape != (1 << len(w), 1 << len(w)):
        raise ValueError("apply_matrix takes 1 to 7 wires and a matching square matrix")
    Uc = np.ascontiguousarray(U, dtype=np.complex128)
    lib().oracle_apply_matrix(_dp(psi.view(np.float64)), n, _ip(w), len(w), _dp(Uc.view(np.float64)))
    return psi


def _op_params(op: Op, params: np.ndarray) -> np.ndarray:
    k = GATE_NPARAMS[op.name]
    return np.asarray(params[op.pidx: op.pidx + k], dtype=np.float64) if k else np.zeros(0)


def op_matrix(op: Op, params: np.ndarray) -> np.ndarray:
    return gate_matrix(op.name, _op_params(op, params), op.matrix, op.inverse)


def apply_op(psi: np.ndarray, n: int, op: Op, params: np.ndarray) -> np.ndarray:
    return apply_matrix(psi, n, op.wires, op_matrix(op, params))


def apply_matrix_at(psi: np.ndarray, n: int, wires: Sequence[int], U: np.ndarray, indices: np.ndarray) -> np.ndarray:
    """Amplitudes ``(U_full psi)[indices]`` for U on ``wires``, one by one (psi unchanged)."""
    _check_state(psi, n)
    w = np.asarray(wires, dtype=np.int32)
    if not 1 <= len(w) <= 7 or U.shape != (1 << len(w), 1 << len(w)):
        raise ValueError("apply_matrix_at takes 1 to 7 wires and a matching square matrix")
    Uc = np.ascontiguousarray(U, dtype=np.complex128)
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    out = np.zeros(len(idx), dtype=np.complex128)
    lib().oracle_apply_matrix_at(_dp(psi.view(np.float64)), n, _ip(w), len(w), _dp(Uc.view(np.float64)),
                                 _up(idx), len(idx), _dp(out.view(np.float64)))
    return out


def apply_op_at(psi: np.ndarray, n: int, op: Op, params: np.ndarray, indices: np.ndarray) -> np.ndarray:
    """Amplitudes ``(U_op psi)[indices]`` computed one by one (psi unchanged)."""
    _check_state(psi, n)
    U = np.ascontiguousarray(op_matrix(op, params))
    w = np.asarray(op.wires, dtype=np.int32)
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    out = np.zeros(len(idx), dtype=np.complex128)
    lib().oracle_apply_matrix_at(_dp(psi.view(np.float64)), n, _ip(w), len(w), _dp(U.view(np.float64)),
                                 _up(idx), len(idx), _dp(out.view(np.float64)))
    return out


def basis_state(n: int, x: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def run_circuit(circuit: Circuit, psi0: Optional[np.ndarray] = None,
                params: Optional[np.ndarray] = None) -> np.ndarray:
    """Applies the circuit's gates in order; returns a new state (|0..0> by default)."""
    n = circuit.n_qubits
    psi = basis_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
    _check_state(psi, n)
    P = np.asarray(circuit.params if params is None else params, dtype=np.float64)
    nops = len(circuit.ops)
    recs = np.zeros((max(nops, 1), 7), dtype=np.int32)
    mats = np.zeros((max(nops, 1), 32), dtype=np.float64)
    for k, op in enumerate(circuit.ops):
        w = list(op.wires) + [0] * (4 - len(op.wires))
        recs[k] = [GATE_ID[op.name], w[0], w[1], w[2], w[3], op.pidx, int(op.inverse)]
        if op.matrix is not None:
            m = np.ascontiguousarray(op.matrix, dtype=np.complex128).reshape(-1)
            mats[k, : 2 * m.size] = m.view(np.float64)
    Pc = np.ascontiguousarray(P if P.size else np.zeros(1))
    rc = lib().oracle_run(_dp(psi.view(np.float64)), n, _ip(recs), nops, _dp(Pc), _dp(mats))
    if rc:
        raise ValueError(f"oracle_run failed at op {-1 - rc}")
    return psi


def norm2(psi: np.ndarray) -> float:
    n = int(psi.size).bit_length() - 1
    _check_state(psi, n)
    return float(lib().oracle_norm2(_dp(psi.view(np.float64)), n))


def expval(psi: np.ndarray, terms: Sequence[Pauli]) -> Tuple[float, np.ndarray]:
    """(sum_w c_w <P_w>, per-word <P_w>) in float64."""
    n = int(psi.size).bit_length() - 1
    _check_state(psi, n)
    c = np.array([t.coeff for t in terms], dtype=np.float64)
    x = np.array([t.x_mask for t in terms], dtype=np.uint64)
    z = np.array([t.z_mask for t in terms], dtype=np.uint64)
    per = np.zeros(len(terms), dtype=np.float64)
    if not len(terms):
        return 0.0, per
    tot = lib().oracle_expval(_dp(psi.view(np.float64)), n, _dp(c), _up(x), _up(z), len(terms), _dp(per))
    return float(tot), per


def energy(circuit: Circuit, terms: Sequence[Pauli], params: Optional[np.ndarray] = None,
           psi0: Optional[np.ndarray] = None) -> float:
    return expval(run_circuit(circuit, psi0, params), terms)[0]


# Shift rules.  A gate whose parameter enters as exp(-i theta K) with K having
# two eigenvalues one apart (RX, RY, RZ, PhaseShift, ControlledPhaseShift and
# each angle of Rot) obeys dE/dtheta = [E(theta + pi/2) - E(theta - pi/2)] / 2.
# CRY's generator P1 (x) Y / 2 has eigenvalues {0, 0, +1/2, -1/2}: two
# frequencies (1/2 and 1), so it takes the four-term rule of Anselmetti et al.
# DoubleExcitation's generator (Y/2 on the pair |0011>, |1100>, 0 elsewhere)
# has the same spectrum and takes the same rule.
# (New J. Phys. 23, 113010, 2021) / Wierichs et al. (Quantum 6, 677, 2022):
#   dE/dtheta = c1 [E(+pi/2) - E(-pi/2)] - c2 [E(+3pi/2) - E(-3pi/2)],
#   c1 = (2 + sqrt 2) / 8, c2 = (2 - sqrt 2) / 8.
_TWO_TERM = {"RX", "RY", "RZ", "PhaseShift", "ControlledPhaseShift", "Rot"}


def param_shift_grad(circuit: Circuit, terms: Sequence[Pauli], psi0: Optional[np.ndarray] = None,
                     params: Optional[np.ndarray] = None) -> np.ndarray:
    """dE/dparams by exact parameter-shift rules (one derivative per parameter
    slot; slots shared by several gates get the sum of their contributions)."""
    P0 = np.asarray(circuit.params if params is None else params, dtype=np.float64)
    g = np.zeros_like(P0)

    def E_with(op_index: int, slot: int, shift: float) -> float:
        # shift only this op's use of the parameter: give it a private copy
        ops = list(circuit.ops)
        op = ops[op_index]
        extra = len(P0)
        pv = np.concatenate([P0, _op_params(op, P0)])
        pv[extra + slot] += shift
        ops[op_index] = Op(op.name, op.wires, extra, op.matrix, op.inverse)
        c = Circuit(circuit.n_qubits, ops, pv)
        return energy(c, terms, psi0=psi0)

    for k, op in enumerate(circuit.ops):
        npar = GATE_NPARAMS[op.name]
        if not npar:
            continue
        for s in range(npar):
            if op.name in _TWO_TERM:
                d = 0.5 * (E_with(k, s, math.pi / 2) - E_with(k, s, -math.pi / 2))
            elif op.name in ("CRY", "DoubleExcitation"):
                c1 = (2.0 + math.sqrt(2.0)) / 8.0
                c2 = (2.0 - math.sqrt(2.0)) / 8.0
                d = c1 * (E_with(k, s, math.pi / 2) - E_with(k, s, -math.pi / 2)) \
                    - c2 * (E_with(k, s, 3 * math.pi / 2) - E_with(k, s, -3 * math.pi / 2))
            else:
                raise ValueError(op.name)
            # the shifted energies already follow the inverse gate's dependence
            g[op.pidx + s] += d
    return g
