"""Fused tile path on the GPU vs the CPU oracle, and fused vs plain."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import MODES, TOL, check_state, gpu_state, max_abs, set_mode

pytestmark = pytest.mark.gpu

CFGS = [None, {"tile_qubits": 5, "low_qubits": 2}, {"tile_qubits": 6, "low_qubits": 4}, {"tile_qubits": 8, "low_qubits": 3},
        {"tile_qubits": 7, "low_qubits": 2, "max_ops": 3}]


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("cfg", CFGS)
@pytest.mark.parametrize("n", [4, 9, 14])
def test_random_circuit_fused(dtype, arith, cfg, n):
    """Random circuits over the whole gate set (several tiles, ragged tile
    shapes, one-tile states), compared amplitude by amplitude."""
    set_mode(arith)
    c = W.random_circuit(n, 150, seed=1000 + n)
    psi0 = W.gaussian_state(n, 2000 + n)
    with gpu_state(n, dtype, psi0) as sv:
        sv.apply(c, fused=True, cfg=cfg)
        check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, len(c.ops))


@pytest.mark.parametrize("dtype,arith", MODES)
def test_ansatz_and_qft_fused_16q(dtype, arith):
    set_mode(arith)
    n = 16
    for c, psi0 in ((W.ansatz(n, 4, 3), oracle.basis_state(n, 0)),
                    (W.qft(n), oracle.basis_state(n, W.basis_index(n, 4))),
                    (W.ghz(n), oracle.basis_state(n, 0))):
        with gpu_state(n, dtype, psi0) as sv:
            sv.apply(c, fused=True)
            check_state(sv.numpy(), oracle.run_circuit(c, psi0), dtype, len(c.ops), c.ops[0].name)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_fused_matches_plain(dtype, arith):
    set_mode(arith)
    n = 17
    c = W.ansatz(n, 3, 11)
    with gpu_state(n, dtype) as a, gpu_state(n, dtype) as b:
        a.apply(c, fused=True)
        b.apply(c, fused=False)
        check_state(a.numpy(), b.numpy(), dtype, 2 * len(c.ops))


@pytest.mark.parametrize("dtype,arith", MODES)
def test_qft_closed_form_20q(dtype, arith):
    """QFT of a basis state: every amplitude is N^-1/2 exp(2 pi i x y / N)."""
    set_mode(arith)
    n = 20
    N = 1 << n
    x = W.basis_index(n, 4)
    with gpu_state(n, dtype, basis=x) as sv:
        sv.apply(W.qft(n), fused=True)
        got = sv.numpy()
    y = np.arange(N, dtype=np.float64)
    ang = 2 * np.pi * ((x * np.arange(N, dtype=np.int64)) % N) / N
    want = np.exp(1j * ang) / np.sqrt(N)
    check_state(got, want, dtype, len(W.qft(n).ops))


def test_df_and_f64_agree_deep_circuit():
    """200 gates: double-float complex128 arithmetic stays within 1e-12 of native float64."""
    n = 12
    c = W.random_circuit(n, 200, seed=99)
    psi0 = W.gaussian_state(n, 98)
    out = {}
    for arith in ("df", "f64"):
        set_mode(arith)
        with gpu_state(n, "c128", psi0) as sv:
            sv.apply(c, fused=False)
            out[arith] = sv.numpy()
    set_mode("df")
    assert max_abs(out["df"], out["f64"]) <= 1e-12
    assert max_abs(out["df"], oracle.run_circuit(c, psi0)) <= 1e-12
