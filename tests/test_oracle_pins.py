"""Pins the CPU oracle to things other than itself (CPU only).

Every check compares the oracle with an independent fact: Pauli algebra, matrix
exponentials of the generators (scipy), tensor-contraction / Kronecker brute
force (numpy), truth tables on basis states, the GHZ and QFT closed forms, the
numpy FFT, and central finite differences.  A plausible slip in the oracle (a
dropped term, a sign, a swapped wire order, a transposed matrix) breaks at
least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG_SEED = 1234

# Pauli matrices as printed in every textbook; they are pinned below by their
# algebra rather than trusted as typed.
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def rand_state(n, seed):
    return W.gaussian_state(n, seed)


def full_operator(n, wires, U):
    """2^n x 2^n operator of U on `wires` by tensor contraction (numpy only).

    The state tensor has one axis per qubit; with C-order reshape axis k is
    qubit n-1-k.  U is reshaped to (2,)*2m with the first listed wire as its
    most significant (first) axis, contracted against the wire axes and the
    result axes moved back into place.  Built column by column from basis
    vectors, it shares nothing with the oracle's index gathering.
    """
    m = len(wires)
    Ut = U.reshape((2,) * (2 * m))
    axes = [n - 1 - w for w in wires]
    N = 1 << n
    F = np.zeros((N, N), dtype=complex)
    for j in range(N):
        e = np.zeros(N, dtype=complex)
        e[j] = 1
        T = e.reshape((2,) * n)
        R = np.tensordot(Ut, T, axes=(list(range(m, 2 * m)), axes))
        R = np.moveaxis(R, list(range(m)), axes)
        F[:, j] = R.reshape(N)
    return F


# ---------------------------------------------------------------------------
# one-qubit gate matrices
# ---------------------------------------------------------------------------

def test_pauli_algebra_pins_xyz():
    x, y, z = (oracle.gate_matrix(g) for g in ("X", "Y", "Z"))
    for s in (x, y, z):
        np.testing.assert_allclose(s @ s, I2, atol=1e-15)
        np.testing.assert_allclose(s, s.conj().T, atol=1e-15)
    np.testing.assert_allclose(x @ y, 1j * z, atol=1e-15)
    np.testing.assert_allclose(y @ z, 1j * x, atol=1e-15)
    np.testing.assert_allclose(z @ x, 1j * y, atol=1e-15)
    # Z is diagonal with Z|0> = |0>, X|0> = |1>: fixes the basis convention
    assert z[0, 0] == 1 and z[1, 1] == -1 and abs(z[0, 1]) == 0
    assert x[1, 0] == 1 and x[0, 0] == 0
    np.testing.assert_allclose(x, X)
    np.testing.assert_allclose(y, Y)
    np.testing.assert_allclose(z, Z)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0, math.pi, 2.5, 5.9])
def test_rotations_are_exponentials_of_paulis(theta):
    for name, s in (("RX", X), ("RY", Y), ("RZ", Z)):
        np.testing.assert_allclose(oracle.gate_matrix(name, [theta]),
                                   scipy.linalg.expm(-0.5j * theta * s), atol=1e-14)


def test_phase_family():
    for phi in (0.2, 1.3, 4.0):
        ps = oracle.gate_matrix("PhaseShift", [phi])
        np.testing.assert_allclose(ps, np.exp(0.5j * phi) * oracle.gate_matrix("RZ", [phi]), atol=1e-14)
        assert ps[0, 0] == 1
    S, T = oracle.gate_matrix("S"), oracle.gate_matrix("T")
    np.testing.assert_allclose(S, oracle.gate_matrix("PhaseShift", [math.pi / 2]), atol=1e-15)
    np.testing.assert_allclose(T, oracle.gate_matrix("PhaseShift", [math.pi / 4]), atol=1e-15)
    np.testing.assert_allclose(S @ S, Z, atol=1e-15)
    np.testing.assert_allclose(T @ T, S, atol=1e-15)


def test_hadamard():
    H = oracle.gate_matrix("H")
    np.testing.assert_allclose(H, (X + Z) / math.sqrt(2), atol=1e-15)
    np.testing.assert_allclose(H @ X @ H, Z, atol=1e-15)
    np.testing.assert_allclose(H @ H, I2, atol=1e-15)


def test_rot_and_additivity():
    a, b = 0.7, 2.1
    np.testing.assert_allclose(oracle.gate_matrix("RZ", [a]) @ oracle.gate_matrix("RZ", [b]),
                               oracle.gate_matrix("RZ", [a + b]), atol=1e-14)
    phi, th, om = 0.4, 1.1, 2.7
    R = oracle.gate_matrix("Rot", [phi, th, om])
    ref = scipy.linalg.expm(-0.5j * om * Z) @ scipy.linalg.expm(-0.5j * th * Y) @ scipy.linalg.expm(-0.5j * phi * Z)
    np.testing.assert_allclose(R, ref, atol=1e-14)
    # with theta = 0 only the two Z rotations remain and they add
    np.testing.assert_allclose(oracle.gate_matrix("Rot", [phi, 0.0, om]), oracle.gate_matrix("RZ", [phi + om]), atol=1e-14)


def test_inverse_is_adjoint():
    for name, p in (("RX", [0.3]), ("Rot", [0.1, 0.2, 0.3]), ("T", []), ("CRY", [0.9]), ("Toffoli", [])):
        U = oracle.gate_matrix(name, p)
        Ui = oracle.gate_matrix(name, p, inverse=True)
        np.testing.assert_allclose(Ui @ U, np.eye(U.shape[0]), atol=1e-14)


def test_user_matrix_passthrough():
    U = W.haar_unitary(4, 5)
    np.testing.assert_allclose(oracle.gate_matrix("U4", matrix=U), U, atol=0)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(4), atol=1e-14)


# ---------------------------------------------------------------------------
# multi-qubit gates on basis states (truth tables fix wire order and bit order)
# ---------------------------------------------------------------------------

def _apply_basis(name, wires, x, n, params=()):
    c = W.Circuit(n).add(name, wires, params)
    return oracle.run_circuit(c, oracle.basis_state(n, x))


def _bit(x, q):
    return (x >> q) & 1


def test_x_flips_bit_q():
    n = 4
    for q in range(n):
        for x in range(1 << n):
            out = _apply_basis("X", (q,), x, n)
            assert out[x ^ (1 << q)] == 1 and np.count_nonzero(out) == 1


def test_cnot_truth_table():
    n = 4
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            for x in range(1 << n):
                out = _apply_basis("CNOT", (c, t), x, n)
                y = x ^ (_bit(x, c) << t)
                assert abs(out[y] - 1) < 1e-15 and np.count_nonzero(out) == 1


def test_toffoli_truth_table():
    n = 4
    for c1, c2, t in ((0, 1, 2), (3, 0, 1), (2, 3, 0), (1, 3, 2)):
        for x in range(1 << n):
            out = _apply_basis("Toffoli", (c1, c2, t), x, n)
            y = x ^ ((_bit(x, c1) & _bit(x, c2)) << t)
            assert abs(out[y] - 1) < 1e-15 and np.count_nonzero(out) == 1


def test_swap_and_phases_on_basis():
    n = 4
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            for x in range(1 << n):
                out = _apply_basis("SWAP", (a, b), x, n)
                y = x & ~((1 << a) | (1 << b)) | (_bit(x, a) << b) | (_bit(x, b) << a)
                assert abs(out[y] - 1) < 1e-15
                out = _apply_basis("CZ", (a, b), x, n)
                assert abs(out[x] - (-1) ** (_bit(x, a) & _bit(x, b))) < 1e-15
                out = _apply_basis("ControlledPhaseShift", (a, b), x, n, [0.77])
                assert abs(out[x] - np.exp(0.77j * (_bit(x, a) & _bit(x, b)))) < 1e-15


def test_two_qubit_identities():
    n = 3
    psi = rand_state(n, 11)

    def run(ops):
        c = W.Circuit(n)
        for name, w in ops:
            c.add(name, w)
        return oracle.run_circuit(c, psi)

    np.testing.assert_allclose(run([("CNOT", (0, 2)), ("CNOT", (0, 2))]), psi, atol=1e-15)
    np.testing.assert_allclose(run([("SWAP", (0, 2))]),
                               run([("CNOT", (0, 2)), ("CNOT", (2, 0)), ("CNOT", (0, 2))]), atol=1e-15)
    np.testing.assert_allclose(run([("CZ", (1, 2))]), run([("H", (2,)), ("CNOT", (1, 2)), ("H", (2,))]), atol=1e-14)
    c = W.Circuit(n).add("ControlledPhaseShift", (1, 2), [math.pi])
    np.testing.assert_allclose(oracle.run_circuit(c, psi), run([("CZ", (1, 2))]), atol=1e-15)


def test_cry_is_exponential_of_controlled_generator():
    th = 1.3
    G = np.kron(P1, Y)  # control is the first (most significant) local wire
    np.testing.assert_allclose(oracle.gate_matrix("CRY", [th]), scipy.linalg.expm(-0.5j * th * G), atol=1e-14)


# ---------------------------------------------------------------------------
# brute force: the oracle's update equals the full operator (tensor contraction)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_apply_matches_tensor_contraction(n):
    rng = np.random.default_rng(RNG_SEED + n)
    psi = rand_state(n, 100 + n)
    for name, m, npar in W.GATES:
        if m > n:
            continue
        for _ in range(3):
            wires = tuple(int(w) for w in rng.permutation(n)[:m])
            params = list(rng.uniform(0, 2 * math.pi, npar))
            mat = W.haar_unitary(1 << m, int(rng.integers(1 << 30))) if name in ("U2", "U4") else None
            inv = bool(rng.integers(2))
            U = oracle.gate_matrix(name, params, mat, inv)
            got = oracle.run_circuit(W.Circuit(n, [W.Op(name, wires, 0 if npar else -1, mat, inv)],
                                               np.asarray(params + [0.0])), psi)
            want = full_operator(n, wires, U) @ psi
            np.testing.assert_allclose(got, want, atol=1e-14, err_msg=f"{name}{wires}")


def test_single_qubit_kron_embedding():
    # qubit q is bit q: the full operator is I_(2^(n-1-q)) (x) U (x) I_(2^q)
    n = 5
    psi = rand_state(n, 7)
    U = W.haar_unitary(2, 8)
    for q in range(n):
        F = np.kron(np.kron(np.eye(1 << (n - 1 - q)), U), np.eye(1 << q))
        got = oracle.apply_matrix(psi.copy(), n, [q], U)
        np.testing.assert_allclose(got, F @ psi, atol=1e-14)


def test_apply_at_matches_full_update():
    n = 8
    psi = rand_state(n, 21)
    idx = np.array([0, 1, 5, 77, 128, 200, 255], dtype=np.uint64)
    for op in (W.Op("H", (3,)), W.Op("U4", (6, 1), -1, W.haar_unitary(4, 3)), W.Op("Toffoli", (0, 7, 4)),
               W.Op("RY", (7,), 0)):
        full = oracle.apply_op(psi.copy(), n, op, np.array([0.42]))
        np.testing.assert_allclose(oracle.apply_op_at(psi, n, op, np.array([0.42]), idx), full[idx.astype(int)],
                                   atol=1e-15)


def test_random_circuits_preserve_norm():
    for n in (3, 7, 10):
        c = W.random_circuit(n, 60, seed=n)
        psi = oracle.run_circuit(c, rand_state(n, n))
        assert abs(oracle.norm2(psi) - 1.0) < 1e-13


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 5, 11])
def test_ghz_closed_form(n):
    psi = oracle.run_circuit(W.ghz(n))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, want, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 10])
def test_qft_basis_closed_form(n):
    N = 1 << n
    for x in sorted({0, 1, N - 1, W.basis_index(n, 4), N // 3}):
        psi = oracle.run_circuit(W.qft(n), oracle.basis_state(n, x))
        y = np.arange(N)
        want = np.exp(2j * np.pi * x * y / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, want, atol=1e-13)


@pytest.mark.parametrize("n", [4, 9, 12])
def test_qft_random_state_is_inverse_fft(n):
    psi0 = rand_state(n, 40 + n)
    psi = oracle.run_circuit(W.qft(n), psi0)
    np.testing.assert_allclose(psi, np.fft.ifft(psi0) * math.sqrt(1 << n), atol=1e-13)


def test_qft_without_swaps_is_bit_reversed():
    n = 6
    N = 1 << n
    psi0 = rand_state(n, 3)
    a = oracle.run_circuit(W.qft(n, swaps=False), psi0)
    b = oracle.run_circuit(W.qft(n), psi0)
    rev = np.array([int(format(i, f"0{n}b")[::-1], 2) for i in range(N)])
    np.testing.assert_allclose(a[rev], b, atol=1e-14)


# ---------------------------------------------------------------------------
# expectation values
# ---------------------------------------------------------------------------

def _pauli_full(n, t):
    M = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        x, z = (t.x_mask >> q) & 1, (t.z_mask >> q) & 1
        s = {(0, 0): I2, (1, 0): X, (0, 1): Z, (1, 1): Y}[(x, z)]
        M = np.kron(M, s)
    return M


def test_expval_matches_kron_pauli_matrices():
    n = 6
    psi = rand_state(n, 9)
    rng = np.random.default_rng(5)
    terms = [W.Pauli(float(rng.normal()), int(rng.integers(1 << n)), int(rng.integers(1 << n))) for _ in range(20)]
    tot, per = oracle.expval(psi, terms)
    for t, v in zip(terms, per):
        want = np.vdot(psi, _pauli_full(n, t) @ psi)
        assert abs(want.imag) < 1e-14
        assert abs(v - want.real) < 1e-14
    assert abs(tot - sum(t.coeff * v for t, v in zip(terms, per))) < 1e-13


def test_expval_eigenstates():
    n = 5
    for x in range(1 << n):
        psi = oracle.basis_state(n, x)
        _, per = oracle.expval(psi, [W.pauli_word(1.0, {q: "Z"}) for q in range(n)])
        np.testing.assert_allclose(per, [(-1) ** ((x >> q) & 1) for q in range(n)])
    plus = np.full(1 << n, 1 / math.sqrt(1 << n), dtype=complex)
    e, _ = oracle.expval(plus, W.tfim(n))
    assert abs(e - 0.5 * n) < 1e-13  # <+|ZZ|+> = 0, <+|X|+> = 1
    e, _ = oracle.expval(oracle.basis_state(n, 0), W.tfim(n))
    assert abs(e - (n - 1)) < 1e-13


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------

def test_param_shift_one_qubit_analytic():
    # <0| RY(t)^dag Z RY(t) |0> = cos t ; <0|RX^dag Z RX|0> = cos t
    for name in ("RY", "RX"):
        for t in (0.1, 1.2, 3.0):
            c = W.Circuit(1).add(name, (0,), [t])
            g = oracle.param_shift_grad(c, [W.pauli_word(1.0, {0: "Z"})])
            assert abs(g[0] + math.sin(t)) < 1e-13
            assert abs(oracle.energy(c, [W.pauli_word(1.0, {0: "Z"})]) - math.cos(t)) < 1e-14


def _fd_grad(c, terms, psi0, h=1e-5):
    g = np.zeros(c.n_params)
    for k in range(c.n_params):
        p = c.params.copy(); p[k] += h
        ep = oracle.energy(c, terms, p, psi0)
        p[k] -= 2 * h
        em = oracle.energy(c, terms, p, psi0)
        g[k] = (ep - em) / (2 * h)
    return g


def test_param_shift_matches_finite_differences_all_gates():
    n = 4
    names = ["RX", "RY", "RZ", "PhaseShift", "Rot", "ControlledPhaseShift", "CRY", "H", "CNOT", "S", "T", "Y", "SWAP",
             "Toffoli", "U2"]
    c = W.random_circuit(n, 40, seed=77, names=names)
    psi0 = rand_state(n, 78)
    terms = W.tfim(n) + [W.pauli_word(0.3, {0: "Y", 2: "X"})]
    g = oracle.param_shift_grad(c, terms, psi0)
    np.testing.assert_allclose(g, _fd_grad(c, terms, psi0), atol=1e-8)


def test_param_shift_ansatz_matches_fd():
    c = W.ansatz(4, 2, seed=6)
    g = oracle.param_shift_grad(c, W.tfim(4))
    np.testing.assert_allclose(g, _fd_grad(c, W.tfim(4), None), atol=1e-8)


# ---------------------------------------------------------------------------
# facts the paper prints
# ---------------------------------------------------------------------------

def test_paper_facts():
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    # 16 bytes per complex128 amplitude: 2^30 amplitudes >= 16 GB, 2^40 ~ 16 TiB
    assert (1 << 30) * 16 / 1e9 >= facts["state_bytes"]["n30_at_least_gb"]
    assert (1 << 40) * 16 / 2 ** 40 == facts["state_bytes"]["n40_approx_tib"]
    # largest gate matrix a kernel applies is 8x8 (Toffoli, CSWAP); DoubleExcitation (Listing 1) is
    # defined by its 16x16 matrix in the oracle, but the GPU path runs it as CNOTs, X and a controlled RY
    assert max(oracle.gate_matrix(g, [0.1] * p, W.haar_unitary(1 << m, 1) if g in ("U2", "U4") else None).shape[0]
               for g, m, p in W.GATES if g != "DoubleExcitation") == facts["max_gate_matrix_dim"]["value"]
    # QFT uses only H and controlled phases (before the final reversal), n H and n(n-1)/2 phases
    for n in (3, 8, 30):
        ops = W.qft(n, swaps=False).ops
        assert {o.name for o in ops} == set(facts["qft_gates"]["gate_kinds"])
        assert sum(o.name == "H" for o in ops) == n
        assert sum(o.name == "ControlledPhaseShift" for o in ops) == n * (n - 1) // 2
        # the R_k angles are pi/2^k, k = control-target distance
        for o in ops:
            if o.name != "H":
                k = abs(o.wires[1] - o.wires[0])
                assert W.qft(n, swaps=False).params[o.pidx] == math.pi / 2 ** k
    # universal-circuit gate count identity 2N^2 = N(N-1) + N(N+1), and the
    # generator's counts and R_k angles (pi / 2^k)
    for N in range(1, 42):
        assert 2 * N * N == N * (N - 1) + N * (N + 1)
    uc = facts["universal_circuit"]
    for N in (2, 5, 30, 38):
        c = W.universal(N)
        assert len(c.ops) == eval(uc["total"], {"N": N})
        assert sum(o.name == "CNOT" for o in c.ops) == eval(uc["cnot"], {"N": N})
        assert sum(o.name == "PhaseShift" for o in c.ops) == eval(uc["rk"], {"N": N})
        ks = {round(math.log2(math.pi / c.params[o.pidx])) for o in c.ops if o.name == "PhaseShift"}
        assert ks <= set(range(1, N + 1))
    # single-gate sweep fixes the CNOT control at 24 (t = 24 uses control 0)
    sw = W.sweep_30q()
    cn = [c for name, c in sw if name.startswith("CNOT")]
    assert all(c.ops[0].wires[0] == facts["cnot_control_24"]["value"] for c in cn if c.ops[0].wires[1] != 24)


def test_cswap_is_three_toffolis():
    """CSWAP(c, a, b) = Toffoli(c, a, b) Toffoli(c, b, a) Toffoli(c, a, b) (swap by three controlled XORs)."""
    n = 5
    psi = rand_state(n, 71)
    for c, a, b in ((0, 1, 2), (4, 0, 3), (2, 4, 1)):
        got = oracle.run_circuit(W.Circuit(n).add("CSWAP", (c, a, b)), psi)
        want = oracle.run_circuit(W.Circuit(n).add("Toffoli", (c, a, b)).add("Toffoli", (c, b, a))
                                  .add("Toffoli", (c, a, b)), psi)
        np.testing.assert_allclose(got, want, atol=1e-15)


def test_double_excitation_definition():
    """DoubleExcitation(theta) rotates |0011>, |1100> (first wire most significant) by theta/2 and fixes
    every other basis state; its angles add, and theta = 2 pi negates the pair."""
    n = 6
    wires = (4, 1, 5, 0)
    th = 0.7
    for x in range(1 << n):
        bits = tuple((x >> w) & 1 for w in wires)
        out = oracle.run_circuit(W.Circuit(n).add("DoubleExcitation", wires, [th]), oracle.basis_state(n, x))
        if bits == (0, 0, 1, 1):
            partner = x ^ sum(1 << w for w in wires)
            assert abs(out[x] - math.cos(th / 2)) < 1e-15 and abs(out[partner] - math.sin(th / 2)) < 1e-15
        elif bits == (1, 1, 0, 0):
            partner = x ^ sum(1 << w for w in wires)
            assert abs(out[x] - math.cos(th / 2)) < 1e-15 and abs(out[partner] + math.sin(th / 2)) < 1e-15
        else:
            assert abs(out[x] - 1.0) < 1e-15 and np.sum(np.abs(out)) - 1.0 < 1e-15
    psi = rand_state(n, 72)
    two = oracle.run_circuit(W.Circuit(n).add("DoubleExcitation", wires, [0.3]).add("DoubleExcitation", wires, [0.5]),
                             psi)
    one = oracle.run_circuit(W.Circuit(n).add("DoubleExcitation", wires, [0.8]), psi)
    np.testing.assert_allclose(two, one, atol=1e-14)
    full = oracle.run_circuit(W.Circuit(n).add("DoubleExcitation", wires, [2 * math.pi]), psi)
    pair = [x for x in range(1 << n) if tuple((x >> w) & 1 for w in wires) in ((0, 0, 1, 1), (1, 1, 0, 0))]
    rest = [x for x in range(1 << n) if x not in pair]
    np.testing.assert_allclose(full[pair], -psi[pair], atol=1e-14)
    np.testing.assert_allclose(full[rest], psi[rest], atol=1e-15)


def test_double_excitation_four_term_shift_matches_finite_differences():
    """The generator's spectrum {0, +-1/2} takes the four-term rule; central differences agree."""
    n = 6
    c = W.Circuit(n)
    for q in range(n):
        c.add("RY", (q,), [0.3 + 0.1 * q])
    c.add("DoubleExcitation", (0, 2, 3, 5), [0.9]).add("CNOT", (1, 4)).add("DoubleExcitation", (5, 4, 1, 0), [-1.3])
    terms = W.tfim(n)
    g = oracle.param_shift_grad(c, terms)
    h = 1e-6
    for k in (n, n + 1):
        p = c.params.copy()
        p[k] += h
        ep = oracle.energy(c, terms, p)
        p[k] -= 2 * h
        em = oracle.energy(c, terms, p)
        assert abs((ep - em) / (2 * h) - g[k]) < 1e-8


@pytest.mark.parametrize("m,wires", [(5, (0, 1, 2, 3, 4)), (5, (4, 3, 2, 1, 0)), (6, (7, 2, 5, 0, 3, 6)),
                                     (7, (1, 0, 7, 6, 3, 5, 2))])
def test_dense_blocks_match_tensor_contraction(m, wires):
    """The general update with 5 to 7 wires (dense blocks) equals the full
    operator built by numpy tensor contraction, for a Haar matrix on ordered
    and scrambled wires."""
    n = 8
    U = W.haar_unitary(1 << m, 77, m)
    psi = rand_state(n, 33 + m)
    want = full_operator(n, wires, U) @ psi
    got = oracle.apply_matrix(psi.copy(), n, wires, U)
    assert np.max(np.abs(got - want)) < 1e-13


def test_dense_block_of_a_product_is_the_product():
    """A 6-wire block that is the Kronecker product of two 3-wire matrices
    equals applying the two factors one after the other (first listed wires
    most significant)."""
    n = 9
    Ua, Ub = W.haar_unitary(8, 78, 1), W.haar_unitary(8, 78, 2)
    wires = (8, 1, 4, 0, 6, 3)
    psi = rand_state(n, 40)
    got = oracle.apply_matrix(psi.copy(), n, wires, np.kron(Ua, Ub))
    want = oracle.apply_matrix(oracle.apply_matrix(psi.copy(), n, wires[3:], Ub), n, wires[:3], Ua)
    assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("n,x", [(5, 0b10110), (7, 0b1001101), (9, 0)])
def test_universal_circuit_on_basis_states(n, x):
    """Every gate of the universal circuit is a phase or a permutation, so a
    basis state stays one basis state times a phase: each layer multiplies by
    e^{i phi} for every qubit whose bit is 1, then the CNOT ladder
    0 -> 1 -> ... -> n-1 replaces bit q+1 by (bit q) xor (bit q+1) in order.
    Tracked with integer bit operations, independently of the oracle."""
    c = W.universal(n)
    state, phase = x, 0.0
    i = 0
    for layer in range(n + 1):
        for q in range(n):
            if (state >> q) & 1:
                phase += c.params[c.ops[i].pidx]
            i += 1
        if layer < n:
            for q in range(n - 1):
                if (state >> q) & 1:
                    state ^= 1 << (q + 1)
            i += n - 1
    want = np.zeros(1 << n, dtype=complex)
    want[state] = np.exp(1j * phase)
    got = oracle.run_circuit(c, oracle.basis_state(n, x))
    assert np.max(np.abs(got - want)) < 1e-13
