"""Small, self-contained GPU workloads for profiling one kernel family at a time.

Usage (for example under ``ncu -k regex:k_fused_reg``)::

    python -m paper_2508_13615_gb300.profile_cases fused 24 c128

Cases: ``fused`` (2-layer RY/RZ/CNOT ansatz on the fused path, applied three
times), ``qft`` (QFT on the fused path, three times), ``expval`` (TFIM
expectation, three times), ``adjoint`` (adjoint gradient of a 2-layer
ansatz), ``gate`` (one dense H per qubit on the plain path), ``u4`` (the
Haar 4x4 gates of the single-gate sweep, U4(t, t+1), on the plain path),
``block`` (a Haar 32x32 block on qubits 0..4 on the tensor cores, three
times; complex64 only), ``batch`` (64 ansatz circuits of 10..N qubits with
their TFIM energies and gradients through the batched driver, twice), ``rz``
(one RZ per qubit) and ``cnot`` (CNOT from the highest qubit to every other
one), both on the plain path.  States start at
|0..0>; the sizes default to 24 qubits so the state (256 MiB complex128)
exceeds the 129 MB L2 while a full ncu capture stays short.
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> None:
    import torch

    import paper_2508_13615_gb300 as L
    import workloads as W

    argv = list(sys.argv[1:] if argv is None else argv)
    mode = argv[0] if argv else "fused"
    n = int(argv[1]) if len(argv) > 1 else 24
    dtype = argv[2] if len(argv) > 2 else "c128"
    sv = L.StateVector(n, dtype)
    sv.set_basis(0)
    if mode == "fused":
        c = W.ansatz(n, 2, 3)
        for _ in range(3):
            sv.apply(c, fused=True)
    elif mode == "qft":
        c = W.qft(n)
        for _ in range(3):
            sv.apply(c, fused=True)
    elif mode == "expval":
        sv.apply(W.ansatz(n, 1, 3), fused=True)
        for _ in range(3):
            sv.expval(W.tfim(n))
    elif mode == "adjoint":
        c = W.ansatz(n, 2, 3)
        sv.apply(c, fused=True)
        sv.adjoint_grad(c, W.tfim(n))
    elif mode == "gate":
        for q in range(n):
            sv.apply_gate("H", (q,))
    elif mode == "block":
        U = W.haar_unitary(32, 91, 0)
        L.lqs_apply_gate(sv.h, "H", (0,))
        for _ in range(3):
            L.lqs_apply_block(sv.h, 5, U)
    elif mode == "rz":
        sv.apply_gate("H", (0,))
        for q in range(n):
            sv.apply_gate("RZ", (q,), (0.3 + 0.1 * q,))
    elif mode == "cnot":
        sv.apply_gate("H", (n - 1,))
        for q in range(n - 1):
            sv.apply_gate("CNOT", (n - 1, q))
    elif mode == "batch":
        # a batch of 64 ansatz circuits of 10..n qubits through the task-queue kernel
        circs = W.batch_circuits(64, 7, n_min=10, n_max=n)
        terms = [W.tfim(c.n_qubits) for c in circs]
        B = L.BatchItems(circs, terms)
        for _ in range(2):
            B.run(dtype)
    elif mode == "u4":
        for _, c in W.sweep_30q(n):
            if c.ops[0].name == "U4":
                sv.apply(c, fused=False)
    else:
        raise SystemExit(f"unknown case {mode}")
    torch.cuda.synchronize()
    sv.close()
    print("ok", mode, n, dtype)


if __name__ == "__main__":
    main()
