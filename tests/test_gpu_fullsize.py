"""Parity at the benchmark's full size: 30 qubits, complex128, the launch
configuration bench.py times (compiled fused segments and Pauli passes).

The oracle cannot run whole 30-qubit circuits in test time, so each check
uses something it can compute at this size:
  * single gates of the sweep: sampled output amplitudes computed one by one
    by the oracle from the same seeded Gaussian input;
  * the QFT of a basis state on the fused path: every sampled amplitude has
    the closed form N^-1/2 exp(2 pi i x y / N), and its TFIM expectation has
    <Z_i Z_i+1> = 0 and <X_q> = cos(2 pi x 2^q / N);
  * the 10-layer ansatz: fused and plain paths agree on sampled amplitudes and
    the norm stays 1.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import set_mode

pytestmark = pytest.mark.gpu

N_Q = 30


@pytest.fixture(scope="module")
def big():
    import torch
    import paper_2508_13615_gb300 as L
    set_mode("df")
    old = L.lqs_jit_info()["mode"]
    L.lqs_set_jit(L.LQS_JIT_ON)  # as bench.py runs: fused segments and Pauli passes compiled
    psi = W.gaussian_state(N_Q, 2)  # the bench's P1 input
    sv = L.StateVector(N_Q, "c128")
    sv.from_numpy(psi)
    saved = sv.tensor.clone()
    yield L, torch, psi, sv, saved
    sv.close()
    L.lqs_set_jit(old)


def sample_indices(seed, count=4096):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 1 << N_Q, size=count, dtype=np.uint64)
    return np.unique(np.concatenate([idx, np.array([0, 1, (1 << N_Q) - 1, 1 << 29, (1 << 24) + 3], dtype=np.uint64)]))


def gather(torch, sv, idx):
    t = torch.as_tensor(idx.astype(np.int64), device=sv.tensor.device)
    return sv.tensor[t].cpu().numpy()


SWEEP_CASES = ["H[0]", "H[29]", "RZ[7]", "CNOT[24,3]", "CNOT[0,24]", "U4[29,0]", "U4[12,13]", "H[17]", "CNOT[24,29]"]


@pytest.mark.parametrize("k", range(len(SWEEP_CASES)), ids=SWEEP_CASES)
def test_sweep_gate_sampled_vs_oracle(big, k):
    which = SWEEP_CASES[k]
    L, torch, psi, sv, saved = big
    c = dict(W.sweep_30q())[which]
    op = c.ops[0]
    sv.tensor.copy_(saved)
    sv.apply(c, fused=False)
    idx = sample_indices(100 + k)
    got = gather(torch, sv, idx)
    want = oracle.apply_op_at(psi, N_Q, op, c.params, idx)
    assert np.max(np.abs(got - want)) <= 1e-12


def test_qft_30q_fused_closed_form_and_tfim(big):
    L, torch, psi, sv, saved = big
    N = 1 << N_Q
    x = W.basis_index(N_Q, 4)
    sv.set_basis(x)
    sv.apply(W.qft(N_Q), fused=True)
    idx = sample_indices(7)
    got = gather(torch, sv, idx)
    ang = 2 * np.pi * ((x * idx.astype(np.int64)) % N) / N
    want = np.exp(1j * ang) / math.sqrt(N)
    assert np.max(np.abs(got - want)) <= 1e-12
    assert abs(sv.norm2() - 1.0) <= 1e-11
    terms = W.tfim(N_Q)
    e, per = sv.expval(terms)
    want_per = [0.0] * (N_Q - 1) + [math.cos(2 * math.pi * ((x << q) % N) / N) for q in range(N_Q)]
    np.testing.assert_allclose(per, want_per, atol=1e-11)
    assert abs(e - sum(t.coeff * w for t, w in zip(terms, want_per))) <= 1e-10


def test_ansatz_30q_fused_matches_plain(big):
    L, torch, psi, sv, saved = big
    c = W.ansatz(N_Q, 10, 3)
    before = L.lqs_jit_info()["launches"]
    sv.set_basis(0)
    sv.apply(c, fused=True)
    assert L.lqs_jit_info()["launches"] > before  # the compiled segments ran
    idx = sample_indices(11)
    fused = gather(torch, sv, idx)
    assert abs(sv.norm2() - 1.0) <= 1e-11
    sv.set_basis(0)
    sv.apply(c, fused=False)
    plain = gather(torch, sv, idx)
    assert np.max(np.abs(fused - plain)) <= 1e-12
