"""Fusion planner checks (host logic, no GPU).

The plan may reorder gates only across gates on disjoint wires.  Executing the
ops segment by segment (original relative order inside a segment) through the
CPU oracle must therefore reproduce the in-order result; and every segment's
tile must hold the low qubits and every non-diagonal target of its gates.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2508_13615_gb300 as L
import workloads as W

DIAG = {"Z", "S", "T", "RZ", "PhaseShift", "CZ", "ControlledPhaseShift"}


def planned_order(c, cfg=None, dtype="c128"):
    nseg, masks, seg_of = L.lqs_plan_fused(c.n_qubits, dtype, c.ops, cfg)
    assert all(0 <= s < nseg for s in seg_of)
    order = sorted(range(len(c.ops)), key=lambda i: (seg_of[i], i))
    return nseg, masks, seg_of, order


def run_in_order(c, order, psi0):
    cc = W.Circuit(c.n_qubits, [c.ops[i] for i in order], c.params)
    return oracle.run_circuit(cc, psi0)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("cfg", [None, {"tile_qubits": 5, "low_qubits": 2}, {"tile_qubits": 4, "low_qubits": 1},
                                 {"tile_qubits": 6, "low_qubits": 3, "max_ops": 5}])
def test_planned_order_reproduces_circuit(seed, cfg):
    n = 9
    # gates that run as one kernel op (DoubleExcitation runs as nine, which the
    # planner may interleave with other gates, so it has no single segment)
    names = [g for g, _, _ in W.GATES if g != "DoubleExcitation"]
    c = W.random_circuit(n, 80, seed=100 + seed, names=names)
    psi0 = W.gaussian_state(n, seed)
    nseg, masks, seg_of, order = planned_order(c, cfg)
    np.testing.assert_allclose(run_in_order(c, order, psi0), oracle.run_circuit(c, psi0), atol=1e-12)


def test_segment_tiles_hold_targets_and_low_qubits():
    n = 20
    c = W.random_circuit(n, 300, seed=5)
    cfg = {"tile_qubits": 8, "low_qubits": 3}
    nseg, masks, seg_of, _ = planned_order(c, cfg)
    for m in masks:
        assert bin(m).count("1") == 8 and (m & 0b111) == 0b111
    for i, op in enumerate(c.ops):
        if op.name in DIAG:
            continue
        m = masks[seg_of[i]]
        targets = op.wires[-1:] if op.name not in ("SWAP", "U4") else op.wires
        if op.name in ("U2", "Rot", "RX", "RY", "H", "X", "Y", "CNOT", "CRY", "Toffoli"):
            targets = op.wires[-1:]
        for t in targets:
            assert (m >> t) & 1, (op.name, op.wires, hex(m))


def test_fusion_cuts_passes_at_least_fourfold():
    for c in (W.ansatz(30, 10, 3), W.qft(30), W.ansatz(24, 8, 6)):
        for dt in ("c128", "c64"):
            nseg = L.lqs_plan_fused(c.n_qubits, dt, c.ops)[0]
            assert len(c.ops) / nseg >= 4, (len(c.ops), nseg)


def test_small_state_is_one_tile():
    c = W.ansatz(6, 3, 1)
    nseg, masks, _, _ = planned_order(c)
    assert nseg == 1 and masks[0] == (1 << 6) - 1
