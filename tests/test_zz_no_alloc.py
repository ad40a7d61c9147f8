"""The allocation-free expectation value (lqs_expval_static).

lqs_expval_static exists for callers that must not allocate device memory when
they measure: hosts whose memory pool owns all device memory, or loops that
cannot pay for the device-wide synchronisation cudaMalloc/cudaFree bring.  It
keeps its partial sums in a fixed scratch array inside the library.  These
tests call it through the C ABI on a raw device pointer, twice in a row (the
second call reuses the same scratch), and check each result against the CPU
oracle and against the handle-based lqs_expval, that the GPU's free memory is
the same before and after the calls, and the empty-Hamiltonian and size-limit
cases.  The file is named to be collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

# per <P_w>: complex128 amplitudes are split into double-float pairs (about
# 2^-47 relative) and accumulated in double-float chains, then float64;
# complex64 amplitudes carry float32 rounding (2^-24 relative)
TOL = {"c128": 1e-12, "c64": 2e-6}


def _call(lib, ptr, n, code, stream, pa, n_terms=None):
    out = ctypes.c_double(np.nan)
    k = pa.n if n_terms is None else n_terms
    per = np.full(max(k, 1), np.nan)
    rc = lib.lqs_expval_static(ctypes.c_void_p(ptr), ctypes.c_int(n), ctypes.c_int(code), ctypes.c_void_p(stream),
                               pa.ptr(), ctypes.c_int(k), ctypes.byref(out),
                               per.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return rc, out.value, per[:k]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_static_expval_matches_oracle_and_handle_expval_twice(dtype):
    import torch

    import paper_2508_13615_gb300 as L
    from paper_2508_13615_gb300 import lqs as B
    n = 14
    c = W.ansatz(n, 2, 12)
    terms = W.tfim(n) + [W.pauli_word(0.4, {0: "Y", 7: "X", 13: "Z"}), W.Pauli(-0.25, (1 << n) - 1, 0b101)]
    with L.StateVector(n, dtype) as sv:
        sv.set_basis(0)
        sv.apply(c, fused=True)
        psi = sv.numpy().astype(np.complex128)
        e_ref, per_ref = sv.expval(terms)
        e_or, per_or = oracle.expval(psi, terms)  # the oracle on the GPU's own state
        ptr, _, code = L.lqs_sv_info(sv.h)
        pa = B.PauliArray(terms)
        lib = ctypes.CDLL(B.LIB_PATH)
        lib.lqs_expval_static.restype = ctypes.c_int
        stream = sv.stream.cuda_stream
        rc, _, _ = _call(lib, ptr, n, code, stream, pa)  # first call: symbol lookup, kernels loaded
        assert rc == 0, L.lqs_last_error()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        scale = sum(abs(t.coeff) for t in terms)
        for _ in range(2):
            rc, e, per = _call(lib, ptr, n, code, stream, pa)
            assert rc == 0, L.lqs_last_error()
            np.testing.assert_allclose(per, per_or, rtol=0, atol=TOL[dtype])
            assert abs(e - e_or) <= TOL[dtype] * scale
            np.testing.assert_allclose(per, per_ref, rtol=0, atol=TOL[dtype])
            assert abs(e - e_ref) <= TOL[dtype] * scale
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the calls"
        assert torch.cuda.memory_allocated() == alloc0
        # no terms: zero, written without touching per_term
        rc, e, _ = _call(lib, ptr, n, code, stream, pa, n_terms=0)
        assert rc == 0 and e == 0.0


def test_static_expval_rejects_too_many_terms():
    import paper_2508_13615_gb300 as L
    n = 8
    with L.StateVector(n, "c128") as sv:
        sv.set_basis(0)
        ptr, _, code = L.lqs_sv_info(sv.h)
        with pytest.raises(L.LqsError) as e:
            L.lqs_expval_static(ptr, n, "c128", [W.pauli_word(1.0, {0: "Z"})] * 65)
        assert e.value.code == L.lqs.LQS_ERR_ARG and "at most 64" in str(e.value)
        # the state is untouched and a valid call still works
        val, per = L.lqs_expval_static(ptr, n, "c128", [W.pauli_word(1.0, {0: "Z"})])
        assert val == pytest.approx(1.0, abs=1e-15) and per[0] == pytest.approx(1.0, abs=1e-15)


def test_static_expval_refuses_a_capturing_stream():
    """On a stream being captured into a CUDA graph the call must refuse
    (LQS_ERR_ARG) before it enqueues anything, so that the capture survives
    and replays; on the same stream outside the capture it works."""
    import torch

    import paper_2508_13615_gb300 as L
    from paper_2508_13615_gb300 import lqs as B
    n = 10
    terms = [W.pauli_word(1.0, {0: "Z"}), W.pauli_word(0.5, {3: "X"})]
    with L.StateVector(n, "c128") as sv:
        sv.set_basis(0)
        ptr, _, code = L.lqs_sv_info(sv.h)
        pa = B.PauliArray(terms)
        lib = ctypes.CDLL(B.LIB_PATH)
        lib.lqs_expval_static.restype = ctypes.c_int
        s = torch.cuda.Stream()
        y = torch.ones(256, device="cuda")
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            rc, _, _ = _call(lib, ptr, n, code, s.cuda_stream, pa)
            y.mul_(2.0)
        assert rc == B.LQS_ERR_ARG and "captured" in L.lqs_last_error()
        g.replay()
        torch.cuda.synchronize()
        assert float(y[0]) == 2.0  # recorded, not run, while capturing; run once by the replay
        rc, e, per = _call(lib, ptr, n, code, s.cuda_stream, pa)
        assert rc == 0, L.lqs_last_error()
        assert e == pytest.approx(1.0, abs=1e-14) and per[1] == pytest.approx(0.0, abs=1e-14)
