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


def _merged_circuit(n, seed):
    """Gates on qubits 0..4 (the block window) interleaved with gates on
    qubits 5..n-1, and every 40 ops a gate joining both sides (it ends a
    run): the fused path must move the outside gates past each run."""
    a = W.random_circuit(5, 160, seed=seed)
    b = W.random_circuit(n - 5, 70, seed=seed + 1)
    c = W.Circuit(n)
    c.params = np.concatenate([a.params, b.params, [0.7, -1.3]])
    off = len(a.params)
    ia = ib = 0
    k = 0
    while ia < len(a.ops) or ib < len(b.ops):
        if ia < len(a.ops) and (k % 3 != 2 or ib >= len(b.ops)):
            c.ops.append(a.ops[ia])
            ia += 1
        elif ib < len(b.ops):
            o = b.ops[ib]
            c.ops.append(W.Op(o.name, tuple(w + 5 for w in o.wires), o.pidx + off if o.pidx >= 0 else -1,
                              o.matrix, o.inverse))
            ib += 1
        k += 1
        if k % 40 == 0:
            c.ops.append(W.Op("CRY", (4, 7 + k % (n - 7)), len(c.params) - 2, None, False))
            c.ops.append(W.Op("CNOT", (9, 2), -1, None, False))
    return c


@pytest.mark.parametrize("n", [14, 17])
def test_fused_path_extracts_tensor_core_blocks(n):
    """lqs_apply_fused on complex64 applies heavy runs on qubits 0..4 as
    tensor-core blocks (and only when allowed); both ways match the oracle."""
    L = _lib()
    c = _merged_circuit(n, 300 + n)
    psi0 = W.gaussian_state(n, 301 + n)
    want = oracle.run_circuit(c, psi0)
    got = {}
    for mode, cfg in (("on", {"tc_blocks": 4}), ("off", {"tc_blocks": -1})):
        with gpu_state(n, "c64", psi0) as sv:
            L.lqs_profile_start()
            sv.apply(c, fused=True, cfg=cfg)
            recs = L.lqs_profile_stop()
            got[mode] = sv.numpy()
        blocks = sum(1 for r in recs if r[0].startswith("k_block_tc"))
        assert (blocks > 0) == (mode == "on"), (mode, blocks)
        assert max_abs(got[mode], want) <= TOL["c64"], mode
    assert max_abs(got["on"], got["off"]) <= TOL["c64"]


def _window_run(c, window, count, seed):
    """`count` Haar U4 gates on neighbouring pairs of `window` (five qubits)."""
    for g in range(count):
        i = (3 * g) % 4
        c.add("U4", (window[i + 1], window[i]), matrix=W.haar_unitary(4, seed, g))


@pytest.mark.parametrize("n", [14, 17, 20])
def test_blocks_on_other_windows(n):
    """Heavy runs on five qubits anywhere in the state (consecutive, spread
    out, the top five) become tensor-core blocks: the fused planner swaps the
    window onto qubits 0..4 around each block (SWAPs it applies as tile
    relabellings) and composes the block from the relabelled gates."""
    L = _lib()
    windows = [(5, 6, 7, 8, 9), (2, 6, 9, 11, n - 2), tuple(range(n - 5, n))]
    c = W.Circuit(n)
    c.add("H", (0,))
    for k, win in enumerate(windows):
        _window_run(c, win, 12, 700 + k)
        c.add("CNOT", (win[0], 0))  # a gate taking a sixth qubit ends the run
    psi0 = W.gaussian_state(n, 710 + n)
    want = oracle.run_circuit(c, psi0)
    got = {}
    for mode, cfg in (("on", None), ("off", {"tc_blocks": -1})):
        with gpu_state(n, "c64", psi0) as sv:
            L.lqs_profile_start()
            sv.apply(c, fused=True, cfg=cfg)
            recs = L.lqs_profile_stop()
            got[mode] = sv.numpy()
        blocks = sum(1 for r in recs if r[0].startswith("k_block_tc"))
        assert blocks == (len(windows) if mode == "on" else 0), (mode, blocks)
        err = max_abs(got[mode], want)
        assert err <= TOL["c64"], (mode, err)
        assert err <= REL * np.max(np.abs(want)) * 4, (mode, err)
