"""Dense 32x32 blocks on the tensor cores (complex64 states) against the
CPU oracle's general matrix update on the same five qubits."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, gpu_state, max_abs

pytestmark = pytest.mark.gpu

# The block acts on qubits 0..4 with qubit q as bit q of the local index; the
# oracle lists the most significant local wire first.
WIRES5 = (4, 3, 2, 1, 0)
# 3xTF32 keeps about float32 accuracy; one TF32 product alone would leave
# errors near 1e-4 of the largest amplitude.
REL = 1e-5


def _lib():
    import paper_2508_13615_gb300 as L
    return L


@pytest.mark.parametrize("n", [12, 13, 16, 20])
def test_haar_block_vs_oracle(n):
    """One Haar-random 32x32 unitary on a Gaussian state: one tile (12
    qubits) up to many tiles per CTA (20 qubits)."""
    L = _lib()
    U = W.haar_unitary(32, 91, n)
    psi0 = W.gaussian_state(n, 90 + n)
    with gpu_state(n, "c64", psi0) as sv:
        L.lqs_apply_block(sv.h, 5, U)
        L.lqs_sv_sync(sv.h)
        got = sv.numpy()
    want = oracle.apply_matrix(psi0.copy(), n, WIRES5, U)
    err = max_abs(got, want)
    assert err <= TOL["c64"]
    assert err <= REL * np.max(np.abs(want)), err


def test_identity_and_permutation_blocks():
    """The identity leaves the state as it was and a permutation matrix
    moves amplitudes only (products with 1 and 0 are exact in every split)."""
    L = _lib()
    n = 14
    psi0 = W.gaussian_state(n, 92).astype(np.complex64)
    perm = np.random.default_rng(93).permutation(32)
    P = np.zeros((32, 32), dtype=np.complex128)
    P[perm, np.arange(32)] = 1.0  # local amplitude c moves to perm[c]
    with gpu_state(n, "c64", psi0) as sv:
        L.lqs_apply_block(sv.h, 5, np.eye(32))
        same = sv.numpy()
        L.lqs_apply_block(sv.h, 5, P)
        moved = sv.numpy()
    assert max_abs(same, psi0) <= 1e-7 * np.max(np.abs(psi0))
    rows = psi0.reshape(-1, 32)
    want = np.empty_like(rows)
    want[:, perm] = rows
    assert max_abs(moved, want.reshape(-1)) <= 1e-7 * np.max(np.abs(psi0))


def test_two_blocks_equal_their_product():
    """U2 after U1 equals the single block U2 U1 (both on the tensor cores)
    and the oracle's two updates."""
    L = _lib()
    n = 15
    U1, U2 = W.haar_unitary(32, 94, 1), W.haar_unitary(32, 94, 2)
    psi0 = W.gaussian_state(n, 95)
    with gpu_state(n, "c64", psi0) as a, gpu_state(n, "c64", psi0) as b:
        L.lqs_apply_block(a.h, 5, U1)
        L.lqs_apply_block(a.h, 5, U2)
        L.lqs_apply_block(b.h, 5, U2 @ U1)
        ga, gb = a.numpy(), b.numpy()
    want = oracle.apply_matrix(oracle.apply_matrix(psi0.copy(), n, WIRES5, U1), n, WIRES5, U2)
    scale = np.max(np.abs(want))
    assert max_abs(ga, want) <= 2 * REL * scale
    assert max_abs(gb, want) <= REL * scale


def test_block_at_24_qubits_sampled():
    """24 qubits (128 MiB, many tiles per CTA): sampled outputs against the
    oracle computed one by one."""
    L = _lib()
    n = 24
    U = W.haar_unitary(32, 96, 0)
    psi0 = W.gaussian_state(n, 97)
    idx = np.unique(np.random.default_rng(98).integers(0, 1 << n, 4096, dtype=np.uint64))
    idx = np.concatenate([idx, np.arange(64, dtype=np.uint64), (1 << n) - 1 - np.arange(64, dtype=np.uint64)])
    with gpu_state(n, "c64", psi0) as sv:
        L.lqs_apply_block(sv.h, 5, U)
        got = sv.numpy()[idx.astype(np.int64)]
    want = oracle.apply_matrix_at(psi0, n, WIRES5, U, idx)
    assert max_abs(got, want) <= REL * np.max(np.abs(psi0)) * 8


def test_block_arguments_are_checked():
    L = _lib()
    U = np.eye(32)
    with gpu_state(14, "c128") as sv:
        with pytest.raises(L.LqsError):
            L.lqs_apply_block(sv.h, 5, U)
    with gpu_state(11, "c64") as sv:
        with pytest.raises(L.LqsError):
            L.lqs_apply_block(sv.h, 5, U)
    with gpu_state(14, "c64") as sv:
        with pytest.raises((L.LqsError, ValueError)):
            L.lqs_apply_block(sv.h, 4, np.eye(16))
        bad = np.eye(32)
        bad[3, 4] = np.nan
        with pytest.raises(L.LqsError):
            L.lqs_apply_block(sv.h, 5, bad)
