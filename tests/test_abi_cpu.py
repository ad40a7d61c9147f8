"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates arguments on the host, and its double-float
conversions meet their stated bounds."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2508_13615_gb300 as L
from paper_2508_13615_gb300 import lqs as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lqs.h")).read()
    return sorted(set(re.findall(r"LQS_API\s+[\w\s\*]+?\b(lqs_\w+)\s*\(", src)))


def test_header_declares_the_core_calls():
    names = declared_symbols()
    for core in ("lqs_sv_alloc", "lqs_apply_gate", "lqs_apply_fused", "lqs_expval", "lqs_adjoint_grad"):
        assert core in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_has_the_same_names():
    for n in declared_symbols():
        assert hasattr(L, n), n


def test_version_and_errors():
    assert L.lqs_version() >= 100
    with pytest.raises(L.LqsError) as e:
        L.lqs_set_arith(7)
    assert e.value.code == B.LQS_ERR_ARG
    assert "arith" in L.lqs_last_error()


def test_alloc_without_device_reports_unsupported():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LqsError) as e:
        L.lqs_sv_alloc(4, "c128")
    assert e.value.code == B.LQS_ERR_UNSUPPORTED


class _Op:
    def __init__(self, name, wires, pidx=-1, matrix=None, inverse=False):
        self.name, self.wires, self.pidx, self.matrix, self.inverse = name, wires, pidx, matrix, inverse


@pytest.mark.parametrize("ops,msg", [
    ([_Op("CNOT", (1, 1))], "repeated wire"),
    ([_Op("H", (9,))], "outside"),
    ([_Op("U2", (0,))], "matrix is NULL"),
])
def test_plan_validates_gates_before_any_work(ops, msg):
    with pytest.raises(L.LqsError) as e:
        L.lqs_plan_fused(8, "c128", ops)
    assert e.value.code == B.LQS_ERR_ARG and msg in str(e.value)


@pytest.mark.parametrize("cfg", [{"tile_qubits": 20}, {"tile_qubits": 10, "low_qubits": 9}, {"arith": 9}])
def test_plan_validates_cfg(cfg):
    with pytest.raises(L.LqsError):
        L.lqs_plan_fused(20, "c128", [_Op("H", (0,))], cfg)


def test_df_split_is_within_two_to_minus_46():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        [1.0, -1.0, 0.5, 2.0 ** -20, np.pi, -np.e, 2.0 ** -103, 2.0 ** 126]])
    x = x[(np.abs(x) >= 2.0 ** -103) & (np.abs(x) < 2.0 ** 127)]  # the documented range
    out = L.lqs_debug_df_roundtrip(x)
    err = np.abs(out - x[:, None])
    big = np.abs(x) >= 2.0 ** -80  # the low float is normal: relative bound
    assert (err[big] / np.abs(x[big])[:, None]).max() <= 2.0 ** -46
    assert err[~big].max() <= 2.0 ** -125  # subnormal low part flushed: absolute bound
    # the store path rounds hi + lo to the nearest double: it equals the exact widening sum
    np.testing.assert_array_equal(out[big, 0], out[big, 1])
    # exact for doubles with at most 47 significant bits
    y = np.round(rng.normal(size=1000) * 2 ** 40) / 2 ** 20
    np.testing.assert_array_equal(L.lqs_debug_df_roundtrip(y)[:, 1], y)


def test_df_flushes_tiny_and_keeps_zero():
    x = np.array([0.0, -0.0, 1e-40, -2.0 ** -104, 2.0 ** -102])
    out = L.lqs_debug_df_roundtrip(x)[:, 1]
    np.testing.assert_array_equal(out[:4], 0.0)
    assert out[4] == 2.0 ** -102


def test_every_handle_call_rejects_a_null_handle_before_any_device_work():
    """Each entry point that takes a state handle returns LQS_ERR_ARG for NULL
    (checked first, so this holds on a machine without a GPU)."""
    R = B._L
    d = ctypes.c_double()
    calls = {
        "lqs_sv_info": lambda: R.lqs_sv_info(None, None, None, None),
        "lqs_sv_set_basis": lambda: R.lqs_sv_set_basis(None, 0),
        "lqs_sv_copy_from_host": lambda: R.lqs_sv_copy_from_host(None, None),
        "lqs_sv_copy_to_host": lambda: R.lqs_sv_copy_to_host(None, None),
        "lqs_sv_copy_to_host_async": lambda: R.lqs_sv_copy_to_host_async(None, None),
        "lqs_sv_sync": lambda: R.lqs_sv_sync(None),
        "lqs_check_bounded_wait": lambda: R.lqs_check_bounded_wait(None),
        "lqs_apply_gate": lambda: R.lqs_apply_gate(None, 3, None, 0, None, 0, 0),
        "lqs_apply_matrix": lambda: R.lqs_apply_matrix(None, None, 0, None),
        "lqs_apply_fused": lambda: R.lqs_apply_fused(None, None, 0, None, 0, None),
        "lqs_apply_block": lambda: R.lqs_apply_block(None, 5, None),
        "lqs_norm2": lambda: R.lqs_norm2(None, ctypes.byref(d)),
        "lqs_expval": lambda: R.lqs_expval(None, None, 0, ctypes.byref(d), None),
        "lqs_adjoint_grad": lambda: R.lqs_adjoint_grad(None, None, 0, None, 0, None, 0, None, None),
        "lqs_sv_distance": lambda: R.lqs_sv_distance(None, None, ctypes.byref(d), ctypes.byref(d)),
        "lqs_autotune_fused": lambda: R.lqs_autotune_fused(None, None, 0, None, 0, 1, None),
    }
    for name, call in calls.items():
        assert call() == B.LQS_ERR_ARG, name


def test_static_expval_and_batch_validate_their_arguments():
    """Argument checks of the allocation-free expectation value and of the
    batched driver, which run before any device work.  The fake device address
    is only ever validated, never used: the test runs only without a GPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import workloads as W
    R = B._L
    d = ctypes.c_double()
    fake = ctypes.c_void_p(256)
    assert R.lqs_expval_static(None, 10, 1, None, None, 0, ctypes.byref(d), None) == B.LQS_ERR_ARG
    many = B.PauliArray(W.tfim(30) + [W.pauli_word(1.0, {q: "Z"}) for q in range(6)])  # 65 words
    assert R.lqs_expval_static(fake, 30, 1, None, many.ptr(), many.n, ctypes.byref(d), None) == B.LQS_ERR_ARG
    assert "at most 64" in L.lqs_last_error()
    outside = B.PauliArray([W.pauli_word(1.0, {31: "Z"})])
    assert R.lqs_expval_static(fake, 30, 1, None, outside.ptr(), outside.n, ctypes.byref(d), None) == B.LQS_ERR_ARG
    assert R.lqs_expval_static(fake, 37, 1, None, None, 0, ctypes.byref(d), None) == B.LQS_ERR_ARG
    assert R.lqs_batch_run(None, 3, 1, None) == B.LQS_ERR_ARG


def test_every_device_wait_goes_through_the_bounded_wait():
    """The only mbarrier poll in the sources is the one inside the bounded wait
    (tile.cuh's mbar_wait, limited by a poll count and the global timer), and
    no kernel source spins on a flag in memory."""
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2508_13615_gb300", "csrc")
    polls = []
    for name in sorted(os.listdir(csrc)):
        if not name.endswith((".cu", ".cuh", ".h")):
            continue
        with open(os.path.join(csrc, name)) as f:
            src = f.read()
        for m in re.finditer(r"mbarrier\.(try_wait|test_wait)", src):
            polls.append(name)
        assert not re.search(r"while\s*\(\s*\*?\s*(volatile|flag|ld_acquire)", src), name
    assert polls == ["tile.cuh"]
    with open(os.path.join(csrc, "tile.cuh")) as f:
        tile = f.read()
    body = tile[tile.index("bool mbar_wait("):]
    body = body[: body.index("\n}\n")]
    assert "kSpinLimit" in body and "kWaitLimitNs" in body and "globaltimer_ns()" in body
