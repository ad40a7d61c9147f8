"""The benchmark's circuit family at the largest sizes the oracle runs whole.

* The layered ansatz (RY and RZ on every qubit, open CNOT ladder) at 20 and 22
  qubits on the compiled fused path, element by element against the oracle's
  whole state, depth at most 200 (complex128 and complex64): the 30- and
  32-qubit benchmark runs use these kernels on the same family.
* The adjoint gradient of the 24-qubit, 8-layer, 384-parameter TFIM circuit
  against central differences (h = 1e-6, complex128) on sampled parameters,
  in the benchmark's launch configuration (compiled segments, compiled reverse
  sweep), and the complex64 gradient against the complex128 one.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import check_state, gpu_state, set_mode

pytestmark = pytest.mark.gpu


@pytest.fixture
def jit_on():
    import paper_2508_13615_gb300 as L
    old = L.lqs_jit_info()["mode"]
    L.lqs_set_jit(L.LQS_JIT_ON)
    before = L.lqs_jit_info()
    yield L, before
    L.lqs_set_jit(old)
    assert L.lqs_jit_info()["failed"] == before["failed"], L.lqs_jit_info()["last_error"]


def ansatz_depth(n, layers):
    """RY, RZ, then a ladder of n-1 CNOTs that each wait for the previous one."""
    return layers * (n + 1)


@pytest.mark.parametrize("dtype,arith", [("c128", "df"), ("c64", "f32")])
@pytest.mark.parametrize("n,layers", [(20, 9), (22, 8)])
def test_ansatz_whole_state_vs_oracle(jit_on, dtype, arith, n, layers):
    L, before = jit_on
    set_mode(arith)
    assert ansatz_depth(n, layers) <= 200
    c = W.ansatz(n, layers, 3)
    want = oracle.run_circuit(c)
    with gpu_state(n, dtype) as sv:
        sv.apply(c, fused=True)
        got = sv.numpy()
    check_state(got, want, dtype, len(c.ops), (n, layers))
    assert L.lqs_jit_info()["launches"] > before["launches"]
    assert abs(np.sum(np.abs(got.astype(np.complex128)) ** 2) - 1.0) <= (1e-12 if dtype == "c128" else 1e-5)


def test_adjoint_24q_against_central_differences(jit_on):
    L, _ = jit_on
    set_mode("df")
    n, layers = 24, 8
    c = W.ansatz(n, layers, 6)
    assert c.n_params == 384
    terms = W.tfim(n)
    ops = L.OpArray(c.ops)
    pa = L.PauliArray(terms)
    h = 1e-6
    sample = [0, 7, 23, 24, 100, 191, 250, 383]
    with gpu_state(n, "c128") as sv:
        sv.apply(c, fused=True)
        g, e = L.lqs_adjoint_grad(sv.h, ops, c.params, pa)
        # the sweep returns the state to |0..0>
        back = sv.numpy()
        assert abs(back[0] - 1.0) <= 1e-12 and float(np.max(np.abs(back[1:]))) <= 1e-12
        for k in sample:
            vals = []
            for sgn in (1, -1):
                p = c.params.copy()
                p[k] += sgn * h
                sv.set_basis(0)
                L.lqs_apply_fused(sv.h, ops, p, None)
                vals.append(L.lqs_expval(sv.h, pa)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            # truncation ~h^2 |E'''| and rounding ~1e-16 |E| / h: 1e-7 is the bound stated for this check
            assert abs(fd - g[k]) <= 1e-7, (k, fd, g[k])
    with gpu_state(n, "c64") as sv:
        sv.apply(c, fused=True)
        g64, e64 = L.lqs_adjoint_grad(sv.h, ops, c.params, pa)
    scale = sum(abs(t.coeff) for t in terms)
    assert abs(e64 - e) <= 2e-5 * scale
    assert float(np.max(np.abs(g64 - g))) <= 5e-4
