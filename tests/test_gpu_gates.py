"""Plain per-gate path on the GPU vs the CPU oracle (element by element)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import MODES, TOL, check_state, gpu_state, max_abs, set_mode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def psi12():
    return W.gaussian_state(12, 1)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_single_gate_suite_12q(psi12, dtype, arith):
    """Every X/H/RZ/RY/U2 target and every ordered CNOT/CZ/SWAP pair, each from a
    fresh copy of the seeded 12-qubit state."""
    set_mode(arith)
    worst = 0.0
    with gpu_state(12, dtype, psi12) as sv:
        for c in W.single_gate_suite_12q(1):
            sv.from_numpy(psi12)
            sv.apply(c, fused=False)
            got = sv.numpy()
            want = oracle.run_circuit(c, psi12)
            err = check_state(got, want, dtype, 1, (c.ops[0].name, c.ops[0].wires))
            worst = max(worst, err)
    print(f"worst {dtype}/{arith}: {worst:.3e}")


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_every_gate_every_size(dtype, arith, n):
    set_mode(arith)
    psi0 = W.gaussian_state(n, 30 + n)
    rng = np.random.default_rng(n)
    with gpu_state(n, dtype, psi0) as sv:
        for name, m, npar in W.GATES:
            if m > n:
                continue
            for trial in range(4):
                wires = tuple(int(w) for w in rng.permutation(n)[:m])
                vals = list(rng.uniform(0, 2 * math.pi, npar))
                mat = W.haar_unitary(1 << m, int(rng.integers(1 << 30))) if name in ("U2", "U4") else None
                c = W.Circuit(n).add(name, wires, vals, matrix=mat, inverse=bool(trial & 1) and name not in ("U2", "U4"))
                sv.from_numpy(psi0)
                sv.apply(c, fused=False)
                check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, 1, (name, wires))


@pytest.mark.parametrize("dtype,arith", MODES)
def test_structured_user_matrices_take_special_kernels(dtype, arith):
    """Diagonal / anti-diagonal / phase U2 and diagonal U4 matrices are lowered to
    the diagonal and permutation classes; results must not change."""
    set_mode(arith)
    n = 7
    psi0 = W.gaussian_state(n, 5)
    mats = [np.diag([np.exp(0.3j), np.exp(-1.1j)]), np.array([[0, 1j], [np.exp(0.7j), 0]]), np.diag([1, np.exp(0.2j)]),
            np.diag(np.exp(1j * np.array([0.1, 0.2, 0.3, 0.4])))]
    with gpu_state(n, dtype, psi0) as sv:
        for m in mats:
            name = "U2" if m.shape[0] == 2 else "U4"
            c = W.Circuit(n).add(name, (5,) if name == "U2" else (6, 2), matrix=m)
            sv.from_numpy(psi0)
            sv.apply(c, fused=False)
            check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, 1, name)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_general_matrix_path_equals_dedicated(dtype, arith):
    """Sec. 3.1's comparison: X and CNOT as dense 2x2 / 4x4 matrices ('general
    approach') give the same state as the dedicated permutation kernels.  The
    permutation moves stored bits; the dense kernel computes 0*a + 1*b, exact in
    float32/float64 and within the 2^-46 double-float split otherwise."""
    tol = 1e-14 if arith == "df" else 0.0
    import paper_2508_13615_gb300 as L
    set_mode(arith)
    n = 10
    psi0 = W.gaussian_state(n, 8)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    CN = np.eye(4, dtype=complex)[[0, 1, 3, 2]]
    with gpu_state(n, dtype, psi0) as a, gpu_state(n, dtype, psi0) as b:
        for t in range(n):
            a.from_numpy(psi0)
            b.from_numpy(psi0)
            a.apply_gate("X", (t,))
            L.lqs_apply_matrix(b.h, (t,), X)
            assert max_abs(a.numpy(), b.numpy()) <= tol
            c = (t + 3) % n
            a.apply_gate("CNOT", (c, t))
            L.lqs_apply_matrix(b.h, (c, t), CN)
            assert max_abs(a.numpy(), b.numpy()) <= tol


def test_validation_errors_leave_state_untouched():
    import paper_2508_13615_gb300 as L
    psi0 = W.gaussian_state(6, 2)
    with gpu_state(6, "c128", psi0) as sv:
        for bad in [("CNOT", (2, 2), ()), ("H", (6,), ()), ("RX", (1,), ()), ("U2", (0,), np.eye(3))]:
            with pytest.raises((L.LqsError, ValueError)):
                sv.apply_gate(*bad)
        np.testing.assert_array_equal(sv.numpy(), psi0)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_cswap_and_double_excitation_every_placement(dtype, arith):
    """The 8x8 and 16x16 gates of the extended set on the plain path, with
    wires below, inside and above the low tile bits, against the oracle."""
    set_mode(arith)
    n = 12
    psi0 = W.gaussian_state(n, 55)
    cases = [("CSWAP", (0, 1, 2), []), ("CSWAP", (11, 0, 6), []), ("CSWAP", (3, 10, 4), []),
             ("DoubleExcitation", (0, 1, 2, 3), [0.4]), ("DoubleExcitation", (11, 2, 7, 0), [-1.1]),
             ("DoubleExcitation", (5, 9, 1, 10), [2.5])]
    for name, wires, p in cases:
        for inv in (False, True):
            c = W.Circuit(n)
            c.ops.append(W.Op(name, wires, 0 if p else -1, None, inv))
            c.params = np.asarray(p if p else [0.0])
            with gpu_state(n, dtype, psi0) as sv:
                sv.apply(c, fused=False)
                check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, 1, (name, wires, inv))


def test_copies_on_other_streams_through_aliased_handles():
    """Handles that share one device buffer but order their calls on different
    streams: an upload on one stream, gates on another, an asynchronous
    read-back on a third, chained by events; the host copy equals the oracle."""
    import torch

    import paper_2508_13615_gb300 as L
    set_mode("df")
    n = 14
    psi0 = W.gaussian_state(n, 9)
    c = W.ansatz(n, 2, 3)
    want = oracle.run_circuit(c, psi0)
    buf = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    s_up, s_run, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    up = L.StateVector(n, "c128", tensor=buf, stream=s_up)
    run = L.StateVector(n, "c128", tensor=buf, stream=s_run)
    down = L.StateVector(n, "c128", tensor=buf, stream=s_down)
    host_in = torch.from_numpy(psi0.astype(np.complex128)).pin_memory().numpy()
    host_out = torch.empty(1 << n, dtype=torch.complex128, pin_memory=True).numpy()
    e_up, e_run = torch.cuda.Event(), torch.cuda.Event()
    L.lqs_sv_copy_from_host(up.h, host_in)
    e_up.record(s_up)
    s_run.wait_event(e_up)
    run.apply(c, fused=False)
    e_run.record(s_run)
    s_down.wait_event(e_run)
    L.lqs_sv_copy_to_host_async(down.h, host_out)
    L.lqs_sv_sync(down.h)
    assert max_abs(host_out, want) <= TOL["c128"]
    for sv in (up, run, down):
        sv.close()
