"""Segment compiler checks that need no GPU: the generated straight-line
kernels compile with NVRTC for sm_103a for every gate class and arithmetic,
structures are shared across angles, and arguments are validated."""
import pytest

import paper_2508_13615_gb300 as L
import workloads as W

ARITHS = [("c128", L.LQS_ARITH_DF), ("c128", L.LQS_ARITH_F64), ("c64", L.LQS_ARITH_AUTO)]


@pytest.mark.parametrize("dtype,arith", ARITHS)
def test_every_gate_class_compiles(dtype, arith):
    """Random circuits over the whole gate set, with controls landing on
    register slots, thread bits and qubits outside the tile."""
    before = L.lqs_jit_info()
    n = 14 if dtype == "c128" else 15
    total = 0
    for seed in (3, 4):
        c = W.random_circuit(n, 90, seed=seed)
        total += L.lqs_jit_precompile(n, dtype, c.ops, c.params, arith)
    after = L.lqs_jit_info()
    assert after["failed"] == before["failed"], after["last_error"]
    assert after["cached"] >= before["cached"]
    assert total >= 0


def test_angles_do_not_change_the_structure():
    """Coefficients are kernel parameters: a circuit that differs only in its
    angles needs no new kernel."""
    a, b = W.ansatz(22, 2, 5), W.ansatz(22, 2, 6)
    assert list(a.params) != list(b.params)
    first = L.lqs_jit_precompile(22, "c128", a.ops, a.params, L.LQS_ARITH_DF)
    assert first >= 1
    cached = L.lqs_jit_info()["cached"]
    assert L.lqs_jit_precompile(22, "c128", b.ops, b.params, L.LQS_ARITH_DF) == 0
    assert L.lqs_jit_info()["cached"] == cached


def test_modes_and_arguments():
    old = L.lqs_jit_info()["mode"]
    try:
        for m in (L.LQS_JIT_OFF, L.LQS_JIT_ON, L.LQS_JIT_AUTO):
            L.lqs_set_jit(m)
            assert L.lqs_jit_info()["mode"] == m
        with pytest.raises(L.LqsError) as e:
            L.lqs_set_jit(7)
        assert e.value.code == L.lqs.LQS_ERR_ARG
    finally:
        L.lqs_set_jit(old)
    c = W.ansatz(14, 1, 1)
    for bad in (dict(n_qubits=0), dict(n_qubits=40), dict(dtype=5), dict(arith=9)):
        kw = dict(n_qubits=14, dtype="c128", arith=L.LQS_ARITH_DF)
        kw.update(bad)
        with pytest.raises((L.LqsError, ValueError)):
            L.lqs_jit_precompile(kw["n_qubits"], kw["dtype"], c.ops, c.params, kw["arith"])


def test_small_states_have_no_segments_to_compile():
    """States that fit one tile never use the register-tile kernel."""
    c = W.ansatz(8, 3, 2)
    assert L.lqs_jit_precompile(8, "c128", c.ops, c.params, L.LQS_ARITH_DF) == 0
