"""Expectation values, norms and adjoint gradients on the GPU vs the oracle."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import MODES, gpu_state, set_mode

pytestmark = pytest.mark.gpu

# Expectation tolerance: terms are bounded by |c_w|; the GPU sums in
# double-float then float64 (complex128) or from float32 amplitudes (complex64).
ETOL = {"c128": 1e-11, "c64": 2e-5}


def random_terms(n, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        x = int(rng.integers(1 << n)) if rng.random() < 0.7 else 0
        z = int(rng.integers(1 << n))
        out.append(W.Pauli(float(rng.normal()), x, z))
    return out


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [1, 3, 9, 15])
def test_expval_random_words(dtype, arith, n):
    set_mode(arith)
    psi = W.gaussian_state(n, 40 + n)
    terms = random_terms(n, 30, n) + W.tfim(n)
    e_ref, per_ref = oracle.expval(psi, terms)
    with gpu_state(n, dtype, psi) as sv:
        e, per = sv.expval(terms)
        assert abs(sv.norm2() - 1.0) <= ETOL[dtype]
    scale = sum(abs(t.coeff) for t in terms)
    assert abs(e - e_ref) <= ETOL[dtype] * scale
    np.testing.assert_allclose(per, per_ref, atol=ETOL[dtype])


@pytest.mark.parametrize("dtype,arith", MODES)
def test_expval_is_deterministic(dtype, arith):
    set_mode(arith)
    n = 18
    with gpu_state(n, dtype) as sv:
        sv.apply(W.ansatz(n, 2, 4), fused=True)
        a = sv.expval(W.tfim(n))
        b = sv.expval(W.tfim(n))
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("dtype,arith", MODES)
def test_adjoint_matches_parameter_shift_12q(dtype, arith):
    """8-layer ansatz at 12 qubits (192 parameters), TFIM observable."""
    set_mode(arith)
    n = 12
    c = W.ansatz(n, 8, 6)
    terms = W.tfim(n)
    g_ref = oracle.param_shift_grad(c, terms)
    e_ref = oracle.energy(c, terms)
    with gpu_state(n, dtype) as sv:
        sv.apply(c, fused=True)
        g, e = sv.adjoint_grad(c, terms)
        back = sv.numpy()
    tol = 1e-10 if dtype == "c128" else 5e-4
    assert abs(e - e_ref) <= tol
    np.testing.assert_allclose(g, g_ref, atol=tol)
    # the sweep returns the state to the circuit's input |0..0>
    assert abs(back[0] - 1.0) <= (1e-12 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_adjoint_all_parametrised_gates(dtype, arith):
    set_mode(arith)
    n = 6
    names = ["RX", "RY", "RZ", "PhaseShift", "Rot", "ControlledPhaseShift", "CRY", "H", "CNOT", "SWAP", "Toffoli", "S",
             "U4", "Y", "DoubleExcitation", "CSWAP"]
    c = W.random_circuit(n, 60, seed=7, names=names)
    psi0 = W.gaussian_state(n, 3)
    terms = W.tfim(n) + [W.pauli_word(0.7, {1: "Y", 4: "X"}), W.pauli_word(-0.2, {0: "Y", 2: "Z", 5: "Y"})]
    g_ref = oracle.param_shift_grad(c, terms, psi0)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True)
        g, e = sv.adjoint_grad(c, terms)
    tol = 1e-10 if dtype == "c128" else 5e-4
    np.testing.assert_allclose(g, g_ref, atol=tol)


def test_adjoint_vs_finite_differences_c128():
    """Central differences, h = 1e-6, on the complex128 GPU path itself."""
    set_mode("df")
    n, h = 10, 1e-6
    c = W.ansatz(n, 3, 21)
    terms = W.tfim(n)
    with gpu_state(n, "c128") as sv:
        sv.apply(c, fused=True)
        g, e = sv.adjoint_grad(c, terms)
        rng = np.random.default_rng(0)
        for k in rng.choice(c.n_params, 12, replace=False):
            vals = []
            for s in (+1, -1):
                p = c.params.copy()
                p[k] += s * h
                cc = W.Circuit(n, c.ops, p)
                sv.set_basis(0)
                sv.apply(cc, fused=True)
                vals.append(sv.expval(terms)[0])
            assert abs((vals[0] - vals[1]) / (2 * h) - g[k]) <= 1e-7


def test_autograd_function():
    import torch
    import paper_2508_13615_gb300 as L
    set_mode("df")
    n = 8
    c = W.ansatz(n, 2, 5)
    terms = W.tfim(n)
    p = torch.tensor(c.params, dtype=torch.float64, requires_grad=True)
    e = L.expval_autograd(p, c, terms)
    e.backward()
    np.testing.assert_allclose(p.grad.numpy(), oracle.param_shift_grad(c, terms), atol=1e-10)
    assert abs(e.item() - oracle.energy(c, terms)) <= 1e-11


@pytest.mark.parametrize("dtype,arith", MODES)
def test_wide_pauli_words_20q(dtype, arith):
    """Words whose X/Y qubits cannot fit a tile take the global pair pass (expectation
    and lambda); the adjoint through such an observable still matches the oracle."""
    set_mode(arith)
    n = 20
    psi = W.gaussian_state(n, 77)
    allx = (1 << n) - 1
    terms = [W.Pauli(0.7, allx, 0), W.Pauli(-0.3, allx, 0b1011), W.Pauli(0.2, 0b1111 << 14, 1 << 3)] + W.tfim(n)
    e_ref, per_ref = oracle.expval(psi, terms)
    with gpu_state(n, dtype, psi) as sv:
        e, per = sv.expval(terms)
    np.testing.assert_allclose(per, per_ref, atol=ETOL[dtype])
    c = W.ansatz(10, 2, 9)
    t10 = [W.Pauli(0.5, (1 << 10) - 1, 0b101)] + W.tfim(10)
    g_ref = oracle.param_shift_grad(c, t10)
    with gpu_state(10, dtype) as sv:
        sv.apply(c, fused=True)
        g, _ = sv.adjoint_grad(c, t10)
    np.testing.assert_allclose(g, g_ref, atol=1e-10 if dtype == "c128" else 5e-4)
