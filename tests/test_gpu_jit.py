"""Compiled segments on the GPU: straight-line kernels against the CPU
oracle and against the register-tile interpreter on the same inputs."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import MODES, TOL, check_state, gpu_state, max_abs, set_mode

pytestmark = pytest.mark.gpu


@pytest.fixture
def jit_on():
    import paper_2508_13615_gb300 as L
    old = L.lqs_jit_info()["mode"]
    L.lqs_set_jit(L.LQS_JIT_ON)
    before = L.lqs_jit_info()
    yield L, before
    L.lqs_set_jit(old)
    after = L.lqs_jit_info()
    assert after["failed"] == before["failed"], after["last_error"]


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,seed", [(14, 21), (16, 22)])
def test_random_circuit_compiled_vs_oracle(jit_on, dtype, arith, n, seed):
    """The whole gate set, 200 gates, from a Gaussian state."""
    L, before = jit_on
    set_mode(arith)
    c = W.random_circuit(n, 200, seed=seed)
    psi0 = W.gaussian_state(n, seed + 100)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True)
        check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, len(c.ops))
    assert L.lqs_jit_info()["launches"] > before["launches"]


@pytest.mark.parametrize("dtype,arith", MODES)
def test_controls_inside_and_outside_the_tile(jit_on, dtype, arith):
    """Controlled gates only: controls fall on register slots, thread bits
    and qubits outside the tile (per-tile predicates)."""
    L, _ = jit_on
    set_mode(arith)
    n = 18
    c = W.random_circuit(n, 160, seed=77, names=["CNOT", "CZ", "CRY", "Toffoli", "ControlledPhaseShift", "H", "RX"])
    psi0 = W.gaussian_state(n, 78)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True)
        check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, len(c.ops))


@pytest.mark.parametrize("dtype,arith", MODES)
def test_compiled_matches_interpreter(dtype, arith):
    """Same circuit, same input: the interpreter (LQS_JIT_OFF) and the
    compiled segments (LQS_JIT_ON) agree to rounding."""
    import paper_2508_13615_gb300 as L
    set_mode(arith)
    n = 20
    out = {}
    old = L.lqs_jit_info()["mode"]
    try:
        for mode in (L.LQS_JIT_OFF, L.LQS_JIT_ON):
            L.lqs_set_jit(mode)
            with gpu_state(n, dtype) as sv:
                sv.apply(W.ansatz(n, 6, 8), fused=True)
                sv.apply(W.qft(n), fused=True)
                out[mode] = sv.numpy()
    finally:
        L.lqs_set_jit(old)
    check_state(out[L.LQS_JIT_ON], out[L.LQS_JIT_OFF], dtype, 2 * (len(W.ansatz(n, 6, 8).ops) + len(W.qft(n).ops)))


def test_compiled_and_interpreted_segments_in_one_call():
    """Consecutive compiled complex128 segments pass the state to each other as
    double-float pairs; a segment the interpreter runs in between reads and
    writes float64.  A circuit whose first part was compiled ahead and whose
    tail was not (automatic mode compiles a structure at its second use) mixes
    both kinds in one call: the result against the oracle."""
    import paper_2508_13615_gb300 as L
    set_mode("df")
    n = 20
    head = W.ansatz(n, 3, 31)
    c = W.ansatz(n, 3, 31)
    for i, q in enumerate((3, 11, 17, 6)):  # a tail whose structures nothing else compiles
        c.add("CRY", (q, (q + 9) % n), (0.4 + i,))
        c.add("Rot", ((q + 4) % n,), (0.1 * i, 0.7, -0.3))
        c.add("RY", ((q + 13) % n,), (1.1 - i,))
    psi0 = W.gaussian_state(n, 77)
    old = L.lqs_jit_info()["mode"]
    try:
        L.lqs_set_jit(L.LQS_JIT_AUTO)
        L.lqs_jit_precompile(n, "c128", head.ops, head.params, L.LQS_ARITH_DF)
        with gpu_state(n, "c128", psi0) as sv:
            L.lqs_profile_start()
            sv.apply(c, fused=True)
            names = [r[0] for r in L.lqs_profile_stop()]
            got = sv.numpy()
    finally:
        L.lqs_set_jit(old)
    assert names.count("k_fused_reg_jit/df") >= 2 and "k_fused_reg/df" in names, names
    check_state(got, oracle.run_circuit(c, psi0), "c128", len(c.ops))


@pytest.mark.parametrize("dtype,arith", MODES)
def test_qft_closed_form_compiled(jit_on, dtype, arith):
    set_mode(arith)
    n = 21
    N = 1 << n
    x = W.basis_index(n, 4)
    with gpu_state(n, dtype, basis=x) as sv:
        sv.apply(W.qft(n), fused=True)
        got = sv.numpy()
    ang = 2 * np.pi * ((x * np.arange(N, dtype=np.int64)) % N) / N
    check_state(got, np.exp(1j * ang) / np.sqrt(N), dtype, len(W.qft(n).ops))


def test_angles_reuse_the_compiled_kernels(jit_on):
    """A second circuit with the same structure and new angles compiles
    nothing and still matches the oracle."""
    L, _ = jit_on
    set_mode("df")
    n = 16
    a, b = W.ansatz(n, 3, 31), W.ansatz(n, 3, 32)
    with gpu_state(n, "c128") as sv:
        sv.apply(a, fused=True)
    compiled = L.lqs_jit_info()["compiled"]
    with gpu_state(n, "c128") as sv:
        sv.apply(b, fused=True)
        err = max_abs(sv.numpy(), oracle.run_circuit(b, oracle.basis_state(n, 0)))
    assert L.lqs_jit_info()["compiled"] == compiled
    assert err <= TOL["c128"]


# ---------------------------------------------------------------------------
# compiled adjoint (reverse sweep over psi and lambda in registers)
# ---------------------------------------------------------------------------
PARAM_GATES = ["RX", "RY", "RZ", "PhaseShift", "Rot", "ControlledPhaseShift", "CRY", "H", "CNOT", "SWAP", "Toffoli",
               "S", "U4", "Y", "CZ", "DoubleExcitation", "CSWAP"]


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,layers", [(13, 6), (15, 4)])
def test_compiled_adjoint_matches_parameter_shift(jit_on, dtype, arith, n, layers):
    """Ansatz (RY, RZ merged into diagonal runs, CNOT renamings) with the TFIM
    observable: every gradient against the oracle's parameter shift."""
    L, before = jit_on
    set_mode(arith)
    c = W.ansatz(n, layers, 6)
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
    assert abs(back[0] - 1.0) <= (1e-12 if dtype == "c128" else 1e-5)
    assert L.lqs_jit_info()["launches"] > before["launches"]


@pytest.mark.parametrize("dtype,arith", MODES)
def test_compiled_adjoint_all_parametrised_gates(jit_on, dtype, arith):
    """Every parametrised gate (RX/RY/RZ, PhaseShift and ControlledPhaseShift
    with P1 generators, decomposed Rot, CRY) among permutations and dense
    gates, from a Gaussian state, with controls and targets inside and
    outside the tile."""
    set_mode(arith)
    n = 13
    c = W.random_circuit(n, 140, seed=17, names=PARAM_GATES)
    psi0 = W.gaussian_state(n, 18)
    terms = W.tfim(n) + [W.pauli_word(0.3, {0: "Y", 7: "X", 12: "Z"})]
    g_ref = oracle.param_shift_grad(c, terms, psi0)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True)
        g, _ = sv.adjoint_grad(c, terms)
    tol = 1e-10 if dtype == "c128" else 5e-4
    np.testing.assert_allclose(g, g_ref, atol=tol)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("with_pi", [False, True])
def test_compiled_adjoint_edge_angles(jit_on, dtype, arith, with_pi):
    """The double-float sweep un-applies RY and H as m00 times a matrix with a
    unit diagonal, so psi and lambda grow by 1/m00 inside a segment and the
    gradient partials come out scaled.  Angles where m00 is small (near pi),
    at the tie |cos| = |sin|, negative and beyond 2 pi; with an angle of
    exactly pi the segment's pivot product leaves float32 range and the
    interpreter sweep runs instead.  Gradients against the oracle's
    parameter shift either way."""
    set_mode(arith)
    n = 13
    angles = [np.pi - 1e-3, -(np.pi - 2e-3), np.pi / 2, 1.2, -2.9, 3 * np.pi + 0.4, 7.0, 1e-9, 2.0, np.pi - 0.05]
    if with_pi:
        angles = angles[:4] + [np.pi] + angles[4:]
    c = W.Circuit(n)
    for i, th in enumerate(angles):
        q = (5 * i) % n
        c.add("RY", (q,), (th,))
        c.add("RZ", ((q + 1) % n,), (0.3 + i,))
        c.add("CNOT", (q, (q + 2) % n))
        if i % 3 == 0:
            c.add("H", ((q + 7) % n,))
    psi0 = W.gaussian_state(n, 515)
    terms = W.tfim(n) + [W.pauli_word(0.4, {2: "Y", 11: "X"})]
    g_ref = oracle.param_shift_grad(c, terms, psi0)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True)
        g, _ = sv.adjoint_grad(c, terms)
    tol = 1e-10 if dtype == "c128" else 5e-4
    np.testing.assert_allclose(g, g_ref, atol=tol)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_compiled_adjoint_matches_interpreter_sweep(dtype, arith):
    """Same circuit and state: gradients of the compiled sweep (LQS_JIT_ON)
    and of the shared-memory sweep (LQS_JIT_OFF)."""
    import paper_2508_13615_gb300 as L
    set_mode(arith)
    n = 18
    c = W.ansatz(n, 5, 9)
    terms = W.tfim(n)
    out = {}
    old = L.lqs_jit_info()["mode"]
    try:
        for mode in (L.LQS_JIT_OFF, L.LQS_JIT_ON):
            L.lqs_set_jit(mode)
            with gpu_state(n, dtype) as sv:
                sv.apply(c, fused=True)
                out[mode] = sv.adjoint_grad(c, terms)
    finally:
        L.lqs_set_jit(old)
    tol = 1e-10 if dtype == "c128" else 5e-4
    np.testing.assert_allclose(out[L.LQS_JIT_ON][0], out[L.LQS_JIT_OFF][0], atol=tol)
    assert abs(out[L.LQS_JIT_ON][1] - out[L.LQS_JIT_OFF][1]) <= tol


# ---------------------------------------------------------------------------
# compiled Pauli passes (expectation values and lambda = H psi)
# ---------------------------------------------------------------------------
def random_words(n, count, seed):
    """Seeded Pauli words of 1..4 factors on any qubits (X, Y and Z land on
    register, thread and outside-tile bits), real coefficients."""
    r = W.splitmix64(seed, 0, 6 * count)
    out = []
    for i in range(count):
        m = 1 + int(r[6 * i] % np.uint64(4))
        word = {}
        for j in range(m):
            q = int(r[6 * i + 1 + j] % np.uint64(n))
            word[q] = "XYZ"[int((r[6 * i + 5] >> np.uint64(2 * j)) % np.uint64(3))]
        out.append(W.pauli_word(float(W.uniforms(seed + 1, i, 1)[0]) - 0.5, word))
    return out


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [14, 17])
def test_compiled_expval_random_words(jit_on, dtype, arith, n):
    L, before = jit_on
    set_mode(arith)
    psi0 = W.gaussian_state(n, 300 + n)
    # words whose X/Y qubits fit a tile (the compiled passes take those)
    terms = [t for t in random_words(n, 60, 31 + n) if bin(int(t.x_mask)).count("1") <= 3] + W.tfim(n)
    e_ref, per_ref = oracle.expval(psi0, terms)
    with gpu_state(n, dtype, psi0) as sv:
        e, per = sv.expval(terms)
    tol = 1e-11 if dtype == "c128" else 2e-5
    np.testing.assert_allclose(per, per_ref, atol=tol)
    assert abs(e - e_ref) <= tol * sum(abs(t.coeff) for t in terms)
    assert L.lqs_jit_info()["launches"] > before["launches"]


@pytest.mark.parametrize("dtype,arith", MODES)
def test_compiled_expval_matches_interpreter(dtype, arith):
    import paper_2508_13615_gb300 as L
    set_mode(arith)
    n = 20
    terms = W.tfim(n) + random_words(n, 20, 77)
    out = {}
    old = L.lqs_jit_info()["mode"]
    try:
        for mode in (L.LQS_JIT_OFF, L.LQS_JIT_ON):
            L.lqs_set_jit(mode)
            with gpu_state(n, dtype) as sv:
                sv.apply(W.ansatz(n, 3, 12), fused=True)
                out[mode] = sv.expval(terms)
    finally:
        L.lqs_set_jit(old)
    tol = 1e-11 if dtype == "c128" else 2e-5
    np.testing.assert_allclose(out[L.LQS_JIT_ON][1], out[L.LQS_JIT_OFF][1], atol=tol)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_compiled_lambda_through_adjoint(jit_on, dtype, arith):
    """lambda = H psi from the compiled passes, checked through gradients of
    an observable with X, Y and Z words on register, thread and outside bits."""
    set_mode(arith)
    n = 14
    c = W.ansatz(n, 3, 21)
    terms = random_words(n, 25, 91) + W.tfim(n)
    terms = [t for t in terms if bin(int(t.x_mask)).count("1") <= 3]
    g_ref = oracle.param_shift_grad(c, terms)
    with gpu_state(n, dtype) as sv:
        sv.apply(c, fused=True)
        g, e = sv.adjoint_grad(c, terms)
    tol = 1e-10 if dtype == "c128" else 5e-4
    np.testing.assert_allclose(g, g_ref, atol=tol)


def test_autotune_choice_is_used_and_correct(jit_on):
    """The tuner returns one of its candidates; lqs_apply_fused without a
    configuration then uses it, and the result matches the oracle."""
    L, _ = jit_on
    set_mode("df")
    n = 17
    c = W.ansatz(n, 3, 41)
    with gpu_state(n, "c128") as sv:
        best = L.lqs_autotune_fused(sv.h, c.ops, c.params, 1)
        assert best["low_qubits"] in (3, 4, 5) and best["max_ops"] in (0, 48)
        sv.set_basis(0)
        sv.apply(c, fused=True)  # no cfg: the tuned one
        err = max_abs(sv.numpy(), oracle.run_circuit(c, oracle.basis_state(n, 0)))
    assert err <= TOL["c128"]
    n_seg = L.lqs_plan_fused(n, "c128", c.ops, best)[0]
    assert n_seg >= 1


@pytest.mark.parametrize("dtype,arith", MODES)
def test_orthogonal_2x2_forms_at_edge_angles(jit_on, dtype, arith):
    """Uncontrolled RY and H run in compiled segments as g times a matrix
    with a unit entry per row, pivoting on m00 or m10 by which is larger.
    Angles on both sides of the switch, at the tie |cos| = |sin|, at the
    zeros of each entry and beyond 2 pi; reflections and a rotation given as
    matrices; targets on register slots, thread bits and outside the tile."""
    L, before = jit_on
    set_mode(arith)
    n = 14
    angles = [0.0, np.pi, -np.pi, np.pi / 2, -np.pi / 2, 1.2, 2.0, -2.9, 3 * np.pi, 7.0, 1e-9, np.pi - 1e-9]
    c = W.Circuit(n)
    for i, th in enumerate(angles * 2):
        q = (3 * i) % n
        c.add("RY", (q,), (th,))
        if i % 3 == 0:
            c.add("H", ((q + 5) % n,))
    for th in (0.3, 2.5, np.pi):
        co, si = np.cos(th / 2), np.sin(th / 2)
        c.add("U2", (int(th * 4) % n,), matrix=np.array([[co, si], [si, -co]], dtype=np.complex128))
    c.add("U2", (9,), matrix=np.array([[0.6, -0.8], [0.8, 0.6]], dtype=np.complex128))
    psi0 = W.gaussian_state(n, 404)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True)
        check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, len(c.ops))
    assert L.lqs_jit_info()["launches"] > before["launches"]


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [13, 16])
def test_universal_circuit_vs_oracle(jit_on, dtype, arith, n):
    """The universal circuit of Sec. 3.2 (2 n^2 phase gates and CNOTs) from a
    Gaussian state, on the fused (compiled) and the plain path."""
    set_mode(arith)
    c = W.universal(n)
    psi0 = W.gaussian_state(n, 500 + n)
    want = oracle.run_circuit(c, psi0)
    for fused in (True, False):
        with gpu_state(n, dtype, psi0) as sv:
            sv.apply(c, fused=fused)
            check_state(sv.numpy(), want, dtype, len(c.ops), fused)
