"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds the inputs only: random numbers, random states, Haar-random
matrices and circuit descriptions (gate names, wires, angles). It contains none
of the simulator's arithmetic -- no gate matrix, no amplitude update, no
expectation value -- so the oracle and the CUDA path stay independent even
though both read their inputs from here.

Conventions (stated once, used everywhere):

* Qubit ``q`` is bit ``q`` of the amplitude index (stride ``2**q``): the paper
  numbers qubits from zero and makes the high qubits the ones that select the
  distant partner (Sec. 2, Fig. 1a/1b), so qubit 0 is the least significant bit.
* A multi-wire gate lists its wires control(s) first, target last (CNOT is
  ``(c, t)``); for a dense 2^m x 2^m matrix the first listed wire is the most
  significant bit of the row/column index.
* Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as
  a counter-based generator: draw ``k`` of stream ``seed`` is
  ``mix64(seed + (k + 1) * 0x9E3779B97F4A7C15)``.  A uniform in [0, 1) is
  ``(x >> 11) * 2**-53``; normals come from the Box-Muller transform; Haar
  unitaries from the QR of a complex Ginibre matrix with the phases of R's
  diagonal divided out (Mezzadri, Notices AMS 54, 2007).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# ---------------------------------------------------------------------------
# SplitMix64 counter-based stream
# ---------------------------------------------------------------------------


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, start_pair: int, count_pairs: int) -> Tuple[np.ndarray, np.ndarray]:
    """``count_pairs`` pairs of independent N(0,1) draws (Box-Muller).

    Pair ``k`` consumes uniforms ``2k`` and ``2k+1`` of the stream; the first is
    mapped to (0, 1] so the logarithm is finite.
    """
    u = uniforms(seed, 2 * start_pair, 2 * count_pairs)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    return r * np.cos(ang), r * np.sin(ang)


def angles(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Angles uniform in [0, 2*pi)."""
    return 2.0 * math.pi * uniforms(seed, start, count)


# ---------------------------------------------------------------------------
# States
# ---------------------------------------------------------------------------

_CHUNK = 1 << 22


def gaussian_state(n_qubits: int, seed: int, out: Optional[np.ndarray] = None,
                   dtype=np.complex128, threads: Optional[int] = None) -> np.ndarray:
    """Seeded i.i.d. complex N(0,1) amplitudes, normalised to unit 2-norm.

    Amplitude ``k`` is ``(z0 + i z1) / ||z||`` from Box-Muller pair ``k`` of
    stream ``seed``.  The norm is accumulated in float64 whatever ``dtype`` is,
    so a complex64 state is the rounding of the complex128 one.  ``out`` (for
    example a pinned host buffer) is filled in place when given.  Large states
    are generated in chunks on a thread pool (numpy releases the GIL).
    """
    N = 1 << n_qubits
    if out is None:
        out = np.empty(N, dtype=dtype)
    if out.shape != (N,) or out.dtype != np.dtype(dtype):
        raise ValueError("out has the wrong shape or dtype")
    nchunks = (N + _CHUNK - 1) // _CHUNK
    sq = np.zeros(nchunks, dtype=np.float64)
    nthreads = max(1, min(threads or 16, os.cpu_count() or 1, nchunks))

    def run(fn) -> None:
        if nthreads == 1:
            for c in range(nchunks):
                fn(c)
        else:
            with ThreadPoolExecutor(nthreads) as ex:
                list(ex.map(fn, range(nchunks)))

    def sumsq(c: int) -> None:
        a, b = c * _CHUNK, min(N, (c + 1) * _CHUNK)
        re, im = normals(seed, a, b - a)
        sq[c] = float(np.dot(re, re) + np.dot(im, im))

    run(sumsq)
    scale = 1.0 / math.sqrt(float(np.sum(sq)))

    def write(c: int) -> None:
        a, b = c * _CHUNK, min(N, (c + 1) * _CHUNK)
        re, im = normals(seed, a, b - a)
        out.real[a:b] = re * scale
        out.imag[a:b] = im * scale

    run(write)
    return out


def basis_index(n_qubits: int, seed: int) -> int:
    """A seeded computational-basis index in [0, 2^n)."""
    return int(splitmix64(seed, 0, 1)[0] >> np.uint64(64 - n_qubits)) if n_qubits > 0 else 0


def haar_unitary(dim: int, seed: int, stream_offset: int = 0) -> np.ndarray:
    """Haar-random ``dim x dim`` unitary (complex128), Mezzadri's QR recipe."""
    re, im = normals(seed, stream_offset, dim * dim)
    z = (re + 1j * im).reshape(dim, dim) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


# ---------------------------------------------------------------------------
# Circuit descriptions
# ---------------------------------------------------------------------------

#: Gate names, their wire count and parameter count.  The numeric id of each is
#: its position in this list (the C ABI uses the same numbering).
GATES: List[Tuple[str, int, int]] = [
    ("X", 1, 0), ("Y", 1, 0), ("Z", 1, 0), ("H", 1, 0), ("S", 1, 0), ("T", 1, 0),
    ("RX", 1, 1), ("RY", 1, 1), ("RZ", 1, 1), ("PhaseShift", 1, 1), ("Rot", 1, 3),
    ("CNOT", 2, 0), ("CZ", 2, 0), ("SWAP", 2, 0), ("ControlledPhaseShift", 2, 1), ("CRY", 2, 1),
    ("Toffoli", 3, 0), ("U2", 1, 0), ("U4", 2, 0), ("CSWAP", 3, 0), ("DoubleExcitation", 4, 1),
]
GATE_ID = {name: i for i, (name, _, _) in enumerate(GATES)}
GATE_WIRES = {name: w for name, w, _ in GATES}
GATE_NPARAMS = {name: p for name, _, p in GATES}


@dataclass
class Op:
    """One gate of a circuit.

    ``pidx`` is the index of the gate's first parameter in the circuit's
    parameter vector (-1 when it has none); ``matrix`` is the caller's unitary
    for U2/U4 (row-major, complex128); ``inverse`` applies the adjoint.
    """
    name: str
    wires: Tuple[int, ...]
    pidx: int = -1
    matrix: Optional[np.ndarray] = None
    inverse: bool = False

    def __post_init__(self) -> None:
        if self.name not in GATE_ID:
            raise ValueError(f"unknown gate {self.name}")
        self.wires = tuple(int(w) for w in self.wires)
        if len(self.wires) != GATE_WIRES[self.name]:
            raise ValueError(f"{self.name} takes {GATE_WIRES[self.name]} wires")


@dataclass
class Circuit:
    n_qubits: int
    ops: List[Op] = field(default_factory=list)
    params: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n_params(self) -> int:
        return int(len(self.params))

    def add(self, name: str, wires: Sequence[int], values: Sequence[float] = (),
            matrix: Optional[np.ndarray] = None, inverse: bool = False) -> "Circuit":
        """Append a gate; its parameter values are appended to ``params``."""
        pidx = -1
        if GATE_NPARAMS[name]:
            if len(values) != GATE_NPARAMS[name]:
                raise ValueError(f"{name} takes {GATE_NPARAMS[name]} parameters")
            pidx = len(self.params)
            self.params = np.concatenate([self.params, np.asarray(values, dtype=np.float64)])
        self.ops.append(Op(name, tuple(wires), pidx, matrix, inverse))
        return self


def ansatz(n_qubits: int, layers: int, seed: int) -> Circuit:
    """Hardware-efficient layered ansatz.

    Layer l: RY(theta_{l,q}) on every qubit, then RZ(phi_{l,q}) on every qubit,
    then the open CNOT ladder (0,1), (1,2), ..., (n-2, n-1).  Parameter flat
    index is ``l*2n + q`` for RY and ``l*2n + n + q`` for RZ; angles are
    U[0, 2pi) drawn in that order from stream ``seed``.
    """
    n = n_qubits
    theta = angles(seed, layers * 2 * n)
    c = Circuit(n)
    c.params = theta.copy()
    for l in range(layers):
        for q in range(n):
            c.ops.append(Op("RY", (q,), l * 2 * n + q))
        for q in range(n):
            c.ops.append(Op("RZ", (q,), l * 2 * n + n + q))
        for q in range(n - 1):
            c.ops.append(Op("CNOT", (q, q + 1)))
    return c


def qft(n_qubits: int, swaps: bool = True) -> Circuit:
    """Quantum Fourier transform from Hadamards and controlled phases (Fig. 5a).

    For j = n-1 down to 0: H on qubit j, then for k = j-1 down to 0 a
    controlled phase of pi / 2^(j-k) with control k and target j.  With
    ``swaps`` the qubit order is reversed at the end (SWAP(i, n-1-i)), so the
    output is the discrete Fourier transform of the input amplitudes.
    """
    c = Circuit(n_qubits)
    vals = []
    for j in range(n_qubits - 1, -1, -1):
        c.ops.append(Op("H", (j,)))
        for k in range(j - 1, -1, -1):
            c.ops.append(Op("ControlledPhaseShift", (k, j), len(vals)))
            vals.append(math.pi / float(1 << (j - k)))
    if swaps:
        for i in range(n_qubits // 2):
            c.ops.append(Op("SWAP", (i, n_qubits - 1 - i)))
    c.params = np.asarray(vals, dtype=np.float64)
    return c


def universal(n_qubits: int) -> Circuit:
    """The N-qubit universal circuit of Sec. 3.2 (Fig. 6a) with phase gates:
    N layers of [R_k on every qubit, then the CNOT ladder 0 -> 1 -> ... ->
    N-1], then R_k on every qubit once more; R_k is the phase gate of angle
    pi / 2^k (PhaseShift), with k = 1 + (layer + qubit) mod N.  That is
    N (N + 1) R_k's and N (N - 1) CNOTs, 2 N^2 gates."""
    n = n_qubits
    c = Circuit(n)
    vals = []
    for layer in range(n + 1):
        for q in range(n):
            c.ops.append(Op("PhaseShift", (q,), len(vals)))
            vals.append(math.pi / float(1 << (1 + (layer + q) % n)))
        if layer < n:
            for q in range(n - 1):
                c.ops.append(Op("CNOT", (q, q + 1)))
    c.params = np.asarray(vals, dtype=np.float64)
    return c


def ghz(n_qubits: int) -> Circuit:
    """H on qubit 0 followed by the CNOT ladder: (|0..0> + |1..1>)/sqrt(2)."""
    c = Circuit(n_qubits)
    c.ops.append(Op("H", (0,)))
    for q in range(n_qubits - 1):
        c.ops.append(Op("CNOT", (q, q + 1)))
    return c


def random_circuit(n_qubits: int, n_ops: int, seed: int,
                   names: Optional[Sequence[str]] = None) -> Circuit:
    """A seeded random circuit over the whole gate set (for parity tests)."""
    names = list(names or [g[0] for g in GATES])
    c = Circuit(n_qubits)
    r = splitmix64(seed, 0, 8 * n_ops)
    vals: List[float] = []
    for i in range(n_ops):
        name = names[int(r[8 * i] % np.uint64(len(names)))]
        m = GATE_WIRES[name]
        if m > n_qubits:
            name, m = "H", 1
        perm = list(range(n_qubits))
        # partial Fisher-Yates for m distinct wires
        for k in range(m):
            j = k + int(r[8 * i + 1 + k] % np.uint64(n_qubits - k))
            perm[k], perm[j] = perm[j], perm[k]
        wires = tuple(perm[:m])
        pidx = -1
        if GATE_NPARAMS[name]:
            pidx = len(vals)
            vals.extend(float(a) for a in angles(seed + 1 + i, GATE_NPARAMS[name]))
        mat = None
        if name == "U2":
            mat = haar_unitary(2, seed * 7919 + i)
        elif name == "U4":
            mat = haar_unitary(4, seed * 7919 + i)
        inverse = bool(int(r[8 * i + 5]) & 1) and name not in ("U2", "U4")
        c.ops.append(Op(name, wires, pidx, mat, inverse))
    c.params = np.asarray(vals, dtype=np.float64)
    return c


# ---------------------------------------------------------------------------
# Observables: sums of Pauli words  H = sum_w c_w P_w
# ---------------------------------------------------------------------------

@dataclass
class Pauli:
    """Pauli word coefficient * prod_q sigma_q.

    Bit q of ``x_mask``/``z_mask`` selects sigma_q: X = (1,0), Z = (0,1),
    Y = (1,1), I = (0,0).
    """
    coeff: float
    x_mask: int
    z_mask: int


def pauli_word(coeff: float, word: dict) -> Pauli:
    """``word`` maps qubit -> 'X' | 'Y' | 'Z'."""
    x = z = 0
    for q, s in word.items():
        if s in ("X", "Y"):
            x |= 1 << q
        if s in ("Z", "Y"):
            z |= 1 << q
    return Pauli(float(coeff), x, z)


def zz_chain(n_qubits: int) -> List[Pauli]:
    """sum_{i=0}^{n-2} Z_i Z_{i+1} (open chain)."""
    return [pauli_word(1.0, {i: "Z", i + 1: "Z"}) for i in range(n_qubits - 1)]


def tfim(n_qubits: int, field_strength: float = 0.5) -> List[Pauli]:
    """Transverse-field Ising model: sum Z_i Z_{i+1} + h * sum X_i (open chain)."""
    return zz_chain(n_qubits) + [pauli_word(field_strength, {i: "X"}) for i in range(n_qubits)]


# ---------------------------------------------------------------------------
# Workload recipes (seeds and shapes of the benchmark configurations)
# ---------------------------------------------------------------------------

def single_gate_suite_12q(seed: int = 1) -> List[Circuit]:
    """12-qubit single-gate suite: X, H, RZ, RY and a Haar U2 on every target,
    CNOT, CZ and SWAP on every ordered pair.  Each case is a one-gate circuit."""
    n = 12
    cases: List[Circuit] = []
    idx = 0
    for name in ("X", "H", "RZ", "RY", "U2"):
        for t in range(n):
            c = Circuit(n)
            if name in ("RZ", "RY"):
                c.add(name, (t,), [float(angles(seed + 1000, 1, idx)[0])])
            elif name == "U2":
                c.add(name, (t,), matrix=haar_unitary(2, seed + 2000, 4 * idx))
            else:
                c.add(name, (t,))
            cases.append(c)
            idx += 1
    for name in ("CNOT", "CZ", "SWAP"):
        for a in range(n):
            for b in range(n):
                if a != b:
                    cases.append(Circuit(n).add(name, (a, b)))
    return cases


def sweep_30q(n: int = 30, seed: int = 2) -> List[Tuple[str, Circuit]]:
    """Single-gate sweep over every target: H(t), RZ(t), CNOT(24, t) (control 0
    when t == 24) and a Haar U4 on (t, t+1 mod n)."""
    out: List[Tuple[str, Circuit]] = []
    th = angles(seed + 100, n)
    ctl = min(24, n - 1)
    for t in range(n):
        out.append((f"H[{t}]", Circuit(n).add("H", (t,))))
    for t in range(n):
        out.append((f"RZ[{t}]", Circuit(n).add("RZ", (t,), [float(th[t])])))
    for t in range(n):
        c = ctl if t != ctl else 0
        out.append((f"CNOT[{c},{t}]", Circuit(n).add("CNOT", (c, t))))
    for t in range(n):
        out.append((f"U4[{t},{(t + 1) % n}]",
                    Circuit(n).add("U4", (t, (t + 1) % n), matrix=haar_unitary(4, seed + 200, 16 * t))))
    return out


def batch_circuits(count: int = 256, seed: int = 7, n_min: int = 10, n_max: int = 20) -> List[Circuit]:
    """Ragged batch: circuit i has n ~ U{n_min..n_max} qubits (10..20 by
    default) and L ~ U{4..12} layers of the ansatz, with parameters from
    stream ``seed + i``."""
    r = splitmix64(seed, 0, 2 * count)
    out = []
    for i in range(count):
        n = n_min + int(r[2 * i] % np.uint64(n_max - n_min + 1))
        L = 4 + int(r[2 * i + 1] % np.uint64(9))
        out.append(ansatz(n, L, seed + i))
    return out
