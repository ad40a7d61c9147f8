"""Edge cases of the GPU path against the oracle: empty circuits, the
smallest states, degenerate observables, circuits without parameters, and a
device-side wait that runs out."""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import MODES, TOL, check_state, gpu_state, max_abs, set_mode

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [1, 14])
def test_empty_circuit_leaves_the_state(dtype, arith, n):
    """No gates: fused and plain paths leave every amplitude as it was."""
    set_mode(arith)
    c = W.Circuit(n)
    psi0 = W.gaussian_state(n, 600 + n).astype(np.complex64 if dtype == "c64" else np.complex128)
    for fused in (True, False):
        with gpu_state(n, dtype, psi0) as sv:
            sv.apply(c, fused=fused)
            np.testing.assert_array_equal(sv.numpy(), psi0)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [1, 2, 3])
def test_smallest_states(dtype, arith, n):
    """States of one to three qubits (one partial tile) through every gate
    that fits, fused and plain."""
    set_mode(arith)
    c = W.random_circuit(n, 60, seed=610 + n)
    psi0 = W.gaussian_state(n, 620 + n)
    want = oracle.run_circuit(c, psi0)
    for fused in (True, False):
        with gpu_state(n, dtype, psi0) as sv:
            sv.apply(c, fused=fused)
            check_state(sv.numpy(), want, dtype, len(c.ops), (n, fused))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_degenerate_observables(dtype):
    """No terms (energy 0), the identity word (its coefficient times the
    norm), a lone Y word on the highest qubit, and a word on every qubit."""
    import paper_2508_13615_gb300 as L
    set_mode("df")
    n = 13
    psi0 = W.gaussian_state(n, 630)
    tol = 1e-11 if dtype == "c128" else 2e-5
    with gpu_state(n, dtype, psi0) as sv:
        e, per = L.lqs_expval(sv.h, [])
        assert e == 0.0 and len(per) == 0
        for terms in ([W.Pauli(0.75, 0, 0)], [W.Pauli(-1.5, 1 << (n - 1), 1 << (n - 1))],
                      [W.Pauli(0.5, (1 << n) - 1, 0b1010101010101)]):
            e, _ = L.lqs_expval(sv.h, terms)
            assert abs(e - oracle.expval(psi0, terms)[0]) <= tol, terms


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_without_parameters(dtype):
    """A circuit with no parametrised gate has an empty gradient, the right
    energy, and the state returns to the input."""
    set_mode("df")
    n = 12
    c = W.ghz(n)
    terms = W.tfim(n)
    with gpu_state(n, dtype, basis=0) as sv:
        sv.apply(c, fused=True)
        g, e = sv.adjoint_grad(c, terms)
        back = sv.numpy()
    assert len(g) == 0
    assert abs(e - oracle.energy(c, terms)) <= (1e-11 if dtype == "c128" else 2e-5)
    assert max_abs(back, oracle.basis_state(n, 0)) <= TOL[dtype]


def test_bounded_wait_gives_up_and_the_state_stays_usable():
    """A kernel waits on a barrier that nothing completes: its bounded wait gives
    up (after 2^22 polls or 2 s of the global timer), the next sync reports LQS_ERR_TIMEOUT once,
    and the same handle then runs a circuit that matches the oracle."""
    import paper_2508_13615_gb300 as L
    set_mode("df")
    n = 12
    c = W.random_circuit(n, 40, seed=620)
    with gpu_state(n, "c128", basis=0) as sv:
        sv.sync()
        t0 = time.perf_counter()
        L.lqs_check_bounded_wait(sv.h)
        with pytest.raises(L.LqsError) as err:
            sv.sync()
        waited = time.perf_counter() - t0
        assert err.value.code == L.lqs.LQS_ERR_TIMEOUT and "gave up" in str(err.value)
        print(f"bounded wait gave up after {waited:.2f} s")
        assert waited <= 30.0
        sv.sync()  # the flag was cleared
        sv.apply(c, fused=True)
        assert max_abs(sv.numpy(), oracle.run_circuit(c)) <= TOL["c128"]
