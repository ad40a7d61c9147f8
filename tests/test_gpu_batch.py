"""Batched circuits (one persistent task-queue launch) vs the oracle, vs one
circuit at a time, repeated calls, and the batch autotuner."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import c64_rel_bound, set_mode

pytestmark = pytest.mark.gpu


def small_batch(seed=3, count=10, nmin=2, nmax=14):
    r = W.splitmix64(seed, 0, 2 * count)
    out = []
    for i in range(count):
        n = nmin + int(r[2 * i] % np.uint64(nmax - nmin + 1))
        L = 1 + int(r[2 * i + 1] % np.uint64(3))
        out.append(W.ansatz(n, L, seed + 10 * i))
    return out


@pytest.mark.parametrize("dtype,arith", [("c128", "df"), ("c128", "f64"), ("c64", "f32")])
def test_batch_matches_oracle(dtype, arith):
    """Energies and gradients of every circuit against the oracle.  complex128:
    1e-10 absolute.  complex64: the float32 rounding bound of the circuit's
    gates (forward for the energy, forward and reverse sweep for the
    gradients) times the observable's coefficient sum."""
    import paper_2508_13615_gb300 as L
    set_mode(arith)
    circs = small_batch() + [W.ansatz(13, 2, 5), W.ansatz(14, 1, 6)]  # several tiles each
    terms = [W.tfim(c.n_qubits) for c in circs]
    e, g = L.lqs_batch_run(circs, terms, dtype)
    for c, t, ei, gi in zip(circs, terms, e, g):
        scale = sum(abs(w.coeff) for w in t)
        if dtype == "c128":
            tol_e = tol_g = 1e-10
        else:
            tol_e = 2 * c64_rel_bound(len(c.ops)) * scale
            tol_g = 4 * c64_rel_bound(2 * len(c.ops)) * scale
        assert abs(ei - oracle.energy(c, t)) <= tol_e, (c.n_qubits, len(c.ops))
        np.testing.assert_allclose(gi, oracle.param_shift_grad(c, t), rtol=0, atol=tol_g)


def test_batch_equals_one_at_a_time():
    import paper_2508_13615_gb300 as L
    set_mode("df")
    circs = small_batch(seed=11, count=16, nmin=8, nmax=16)
    terms = [W.tfim(c.n_qubits) + [W.pauli_word(0.3, {0: "Y", 1: "Y"})] for c in circs]
    e, g = L.lqs_batch_run(circs, terms, "c64")
    for c, t, ei, gi in zip(circs, terms, e, g):
        with L.StateVector(c.n_qubits, "c64") as sv:
            sv.set_basis(0)
            sv.apply(c, fused=True)
            g1, e1 = sv.adjoint_grad(c, t)
        scale = sum(abs(w.coeff) for w in t)
        assert abs(ei - e1) <= 4 * c64_rel_bound(len(c.ops)) * scale
        np.testing.assert_allclose(gi, g1, rtol=0, atol=8 * c64_rel_bound(2 * len(c.ops)) * scale)


def test_batch_energy_only_and_ragged_edge_cases():
    import paper_2508_13615_gb300 as L
    set_mode("df")
    circs = [W.ansatz(1, 1, 1), W.Circuit(3), W.ghz(5), W.qft(6)]  # one qubit, no gates, no parameters
    terms = [[W.pauli_word(1.0, {0: "Z"})], W.tfim(3), W.zz_chain(5), W.tfim(6)]
    e, g = L.lqs_batch_run(circs, terms, "c128", grads=False)
    for c, t, ei in zip(circs, terms, e):
        assert abs(ei - oracle.energy(c, t)) <= 1e-12


@pytest.mark.parametrize("dtype,arith", [("c128", "df"), ("c64", "f32")])
def test_batch_multi_tile_circuits_match_oracle(dtype, arith):
    """Circuits of 13-16 qubits span 2-32 tiles: their tiles run as separate
    tasks that wait for the previous pass of their own circuit."""
    import paper_2508_13615_gb300 as L
    set_mode(arith)
    circs = [W.ansatz(16, 2, 71), W.ansatz(13, 3, 72), W.ansatz(15, 1, 73), W.ansatz(11, 2, 74)]
    circs.append(W.random_circuit(14, 60, seed=75, names=["RX", "RY", "RZ", "CNOT", "H", "CRY", "ControlledPhaseShift",
                                                           "SWAP", "PhaseShift"]))
    terms = [W.tfim(c.n_qubits) + [W.pauli_word(0.2, {0: "Y", 1: "X"})] for c in circs]
    e, g = L.lqs_batch_run(circs, terms, dtype)
    for c, t, ei, gi in zip(circs, terms, e, g):
        scale = sum(abs(w.coeff) for w in t)
        tol_e = 1e-10 if dtype == "c128" else 2 * c64_rel_bound(len(c.ops)) * scale
        tol_g = 1e-10 if dtype == "c128" else 4 * c64_rel_bound(2 * len(c.ops)) * scale
        assert abs(ei - oracle.energy(c, t)) <= tol_e, (c.n_qubits, ei)
        np.testing.assert_allclose(gi, oracle.param_shift_grad(c, t), rtol=0, atol=tol_g)


def test_batch_repeated_calls_are_bit_identical():
    """Partial sums are reduced in a fixed order whatever the task schedule."""
    import paper_2508_13615_gb300 as L
    set_mode("df")
    circs = small_batch(seed=21, count=24, nmin=9, nmax=16)
    terms = [W.tfim(c.n_qubits) for c in circs]
    e1, g1 = L.lqs_batch_run(circs, terms, "c64")
    e2, g2 = L.lqs_batch_run(circs, terms, "c64")
    np.testing.assert_array_equal(e1, e2)
    for a, b in zip(g1, g2):
        np.testing.assert_array_equal(a, b)


def test_batch_autotune_keeps_a_shape_per_qubit_count():
    import paper_2508_13615_gb300 as L
    set_mode("df")
    circs = [W.ansatz(14, 2, 81), W.ansatz(14, 3, 82), W.ansatz(13, 2, 83), W.ansatz(10, 2, 84)]
    terms = [W.tfim(c.n_qubits) for c in circs]
    tuned = L.lqs_batch_autotune(circs, terms, "c64", repeats=1)
    assert tuned == 2  # 13 and 14 qubits span several tiles; 10 qubits is one tile
    e, g = L.lqs_batch_run(circs, terms, "c64")
    for c, t, ei, gi in zip(circs, terms, e, g):
        scale = sum(abs(w.coeff) for w in t)
        assert abs(ei - oracle.energy(c, t)) <= 2 * c64_rel_bound(len(c.ops)) * scale
        np.testing.assert_allclose(gi, oracle.param_shift_grad(c, t), rtol=0,
                                   atol=4 * c64_rel_bound(2 * len(c.ops)) * scale)
