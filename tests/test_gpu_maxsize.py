"""Parity at the largest states these tests place on one GPU: 33 qubits in
complex64 and 32 qubits in complex128 (64 GiB each; amplitude indices of
33 bits), with every gate class on the highest qubits.

The oracle cannot hold such a state, so the circuit is built to have an
exact factorised form.  A layer RY(theta_q), RZ(phi_q) on every qubit makes
the product state (x)_q u_q; a random circuit over the whole gate set then
acts only on a set S of six qubits (the two highest, qubits 0, 1, 5 and 13).
Gates on S leave the other factors alone, so the output is

    psi = phi_S (x) (x)_{q not in S} u_q,

with phi_S the oracle's six-qubit run of the same layer and random circuit
on S.  Every sampled amplitude is phi_S[x restricted to S] times the product
of u_q[x_q]; the expectation of a Pauli word is the product of its parts'
expectations on phi_S and on each u_q; a gradient follows by the product
rule from the oracle's parameter-shift gradients of those parts.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import set_mode

# gates whose gradients the adjoint sweep supports, with unparametrised ones among them
PARAM_GATES = ["RX", "RY", "RZ", "PhaseShift", "Rot", "ControlledPhaseShift", "CRY", "H", "CNOT", "SWAP",
               "Toffoli", "S", "U4", "Y", "CZ", "DoubleExcitation", "CSWAP"]

CASES = [("c64", 33), ("c128", 32)]
# rounding is relative to the amplitudes a gate combines; on this state they
# are bounded by the scale s(x) below, so the bound is tol * s(x)
REL_TOL = {"c64": 2e-5, "c128": 1e-12}
E_TOL = {"c64": 2e-5, "c128": 1e-11}
G_TOL = {"c64": 5e-4, "c128": 1e-10}


def s_set(n):
    return [0, 1, 5, min(13, n - 3), n - 2, n - 1]


def build(n, seed, names=None, n_ops=40):
    """(big circuit on n qubits, circuit on the six qubits of S, per-qubit
    one-qubit circuits, S)."""
    S = s_set(n)
    th = W.angles(seed, 2 * n)
    big = W.Circuit(n)
    for q in range(n):
        big.add("RY", (q,), [float(th[2 * q])])
        big.add("RZ", (q,), [float(th[2 * q + 1])])
    small = W.Circuit(len(S))
    for i, q in enumerate(S):
        small.add("RY", (i,), [float(th[2 * q])])
        small.add("RZ", (i,), [float(th[2 * q + 1])])
    rc = W.random_circuit(len(S), n_ops, seed + 1, names=names)
    for op in rc.ops:
        k = W.GATE_NPARAMS[op.name]
        vals = rc.params[op.pidx: op.pidx + k] if k else ()
        big.add(op.name, tuple(S[w] for w in op.wires), vals, op.matrix, op.inverse)
        small.add(op.name, op.wires, vals, op.matrix, op.inverse)
    one = {q: W.Circuit(1).add("RY", (0,), [float(th[2 * q])]).add("RZ", (0,), [float(th[2 * q + 1])])
           for q in range(n) if q not in S}
    return big, small, one, S


def local_mask(mask, S):
    return sum(((mask >> q) & 1) << i for i, q in enumerate(S))


def factor_expvals(terms, phi, u, S):
    """Per word: (its expectation on phi_S, {q: its expectation on u_q})."""
    out = []
    for t in terms:
        a = oracle.expval(phi, [W.Pauli(1.0, local_mask(t.x_mask, S), local_mask(t.z_mask, S))])[0]
        b = {q: oracle.expval(uq, [W.Pauli(1.0, (t.x_mask >> q) & 1, (t.z_mask >> q) & 1)])[0]
             for q, uq in u.items() if ((t.x_mask | t.z_mask) >> q) & 1}
        out.append((a, b))
    return out


def observables(n):
    S = s_set(n)
    return W.tfim(n) + [W.pauli_word(0.3, {n - 1: "Y", 3: "X"}),
                        W.pauli_word(-0.7, {0: "Z", n - 1: "Z", n - 2: "X"}),
                        W.pauli_word(0.2, {S[3]: "Y", S[3] - 1: "Y", n - 1: "X"})]


def reference_energy(terms, phi, u, S):
    """(energy, per-word expectations) from the factors."""
    per = [a * float(np.prod(list(b.values()))) for a, b in factor_expvals(terms, phi, u, S)]
    return sum(t.coeff * w for t, w in zip(terms, per)), per


def reference_gradient(c, small, one, S, terms, phi, u):
    """dE/dparams of the big circuit by the product rule over the factors: the
    six-qubit part's parameters (its layer angles, then the random circuit's),
    then each u_q's two angles."""
    n = c.n_qubits
    g = np.zeros(c.n_params)
    small_to_big = [2 * S[i // 2] + (i % 2) for i in range(2 * len(S))] + list(range(2 * n, c.n_params))
    for t, (a, b) in zip(terms, factor_expvals(terms, phi, u, S)):
        rest = float(np.prod(list(b.values())))
        word = W.Pauli(1.0, local_mask(t.x_mask, S), local_mask(t.z_mask, S))
        g[small_to_big] += t.coeff * rest * oracle.param_shift_grad(small, [word])
        for q in b:
            dq = oracle.param_shift_grad(one[q], [W.Pauli(1.0, (t.x_mask >> q) & 1, (t.z_mask >> q) & 1)])
            others = float(np.prod([v for p, v in b.items() if p != q]))
            g[2 * q: 2 * q + 2] += t.coeff * a * others * dq
    return g


@pytest.fixture(scope="module", params=CASES, ids=[f"{d}-{n}q" for d, n in CASES])
def big(request):
    import torch
    import paper_2508_13615_gb300 as L
    dtype, n = request.param
    set_mode("df")
    old = L.lqs_jit_info()["mode"]
    L.lqs_set_jit(L.LQS_JIT_ON)  # as bench.py runs
    sv = L.StateVector(n, dtype)
    yield L, torch, dtype, n, sv
    sv.close()
    sv.tensor = None  # release the 64 GiB before the next case allocates its own
    L.lqs_set_jit(old)
    torch.cuda.empty_cache()


def samples(n, seed, count=4096):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 1 << n, size=count, dtype=np.uint64)
    top = (1 << n) - 1
    return np.unique(np.concatenate([idx, np.array([0, 1, top, top - 1, 1 << (n - 1), (1 << 32) - 1,
                                                    (1 << (n - 1)) | 0x2023], dtype=np.uint64)]))


def expected_amplitudes(idx, phi, u, S):
    li = np.zeros(idx.size, dtype=np.int64)
    for i, q in enumerate(S):
        li |= ((idx >> np.uint64(q)) & np.uint64(1)).astype(np.int64) << i
    amp = phi[li].astype(np.complex128)
    scale = np.full(idx.size, np.max(np.abs(phi)))
    for q, uq in u.items():
        amp = amp * uq[((idx >> np.uint64(q)) & np.uint64(1)).astype(np.int64)]
        scale = scale * np.max(np.abs(uq))
    return amp, scale


@pytest.mark.gpu
@pytest.mark.parametrize("fused", [True, False], ids=["fused", "plain"])
def test_top_qubits_sampled_amplitudes_and_expvals(big, fused):
    L, torch, dtype, n, sv = big
    c, small, one, S = build(n, 4100 + n)
    phi = oracle.run_circuit(small)
    u = {q: oracle.run_circuit(cq) for q, cq in one.items()}
    sv.set_basis(0)
    before = L.lqs_jit_info()["launches"]
    sv.apply(c, fused=fused)
    if fused:
        assert L.lqs_jit_info()["launches"] > before  # the compiled segments ran
    idx = samples(n, 5 + n)
    got = sv.tensor[torch.as_tensor(idx.astype(np.int64), device=sv.tensor.device)].cpu().numpy()
    want, scale = expected_amplitudes(idx, phi, u, S)
    err = np.abs(got.astype(np.complex128) - want)
    assert np.max(err) <= {"c64": 2e-5, "c128": 1e-12}[dtype]
    assert np.max(err / scale) <= REL_TOL[dtype], int(idx[np.argmax(err / scale)])
    assert abs(sv.norm2() - 1.0) <= (1e-11 if dtype == "c128" else 2e-5)
    terms = observables(n)
    e, per = sv.expval(terms)
    e_ref, want_per = reference_energy(terms, phi, u, S)
    np.testing.assert_allclose(per, want_per, atol=E_TOL[dtype])
    assert abs(e - e_ref) <= E_TOL[dtype] * sum(abs(t.coeff) for t in terms)


@pytest.mark.gpu
def test_top_qubits_adjoint_gradient(big):
    L, torch, dtype, n, sv = big
    c, small, one, S = build(n, 4300 + n, names=PARAM_GATES, n_ops=30)
    phi = oracle.run_circuit(small)
    u = {q: oracle.run_circuit(cq) for q, cq in one.items()}
    terms = observables(n)
    e_ref, _ = reference_energy(terms, phi, u, S)
    g_ref = reference_gradient(c, small, one, S, terms, phi, u)
    sv.set_basis(0)
    sv.apply(c, fused=True)
    g, e = sv.adjoint_grad(c, terms)
    assert abs(e - e_ref) <= E_TOL[dtype] * sum(abs(t.coeff) for t in terms)
    np.testing.assert_allclose(g, g_ref, atol=G_TOL[dtype])
    # the sweep returns the state to its input |0...0>
    idx = samples(n, 9)
    back = sv.tensor[torch.as_tensor(idx.astype(np.int64), device=sv.tensor.device)].cpu().numpy()
    want = (idx == 0).astype(np.complex128)
    assert np.max(np.abs(back - want)) <= (1e-12 if dtype == "c128" else 2e-5)


@pytest.mark.parametrize("names,n_ops,seed", [(None, 40, 71), (PARAM_GATES, 30, 72)])
def test_factorised_reference_against_the_whole_oracle(names, n_ops, seed):
    """The factorised expected values used above, at 10 qubits where the
    oracle runs the whole circuit: every amplitude, every word's expectation
    and every parameter's gradient."""
    n = 10
    c, small, one, S = build(n, seed, names=names, n_ops=n_ops)
    phi = oracle.run_circuit(small)
    u = {q: oracle.run_circuit(cq) for q, cq in one.items()}
    psi = oracle.run_circuit(c)
    idx = np.arange(1 << n, dtype=np.uint64)
    want, scale = expected_amplitudes(idx, phi, u, S)
    assert np.max(np.abs(psi - want)) <= 1e-14
    assert np.all(np.abs(want) <= scale * (1 + 1e-12))
    terms = observables(n)
    e_ref, per_ref = reference_energy(terms, phi, u, S)
    e, per = oracle.expval(psi, terms)
    np.testing.assert_allclose(per_ref, per, atol=1e-13)
    assert abs(e_ref - e) <= 1e-12
    if names is not None:
        np.testing.assert_allclose(reference_gradient(c, small, one, S, terms, phi, u),
                                   oracle.param_shift_grad(c, terms), atol=1e-12)
