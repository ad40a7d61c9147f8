"""The allocation-free expectation value (lqs_expval_static) agrees with lqs_expval.

lqs_expval_static exists for callers that must not allocate device memory when
they measure (for example while a stream is being captured into a graph): it
keeps its partial sums in a fixed scratch array inside the library.  This test
calls it through the C ABI on a raw device pointer, twice in a row (the second
call reuses the same scratch), and compares with the handle-based call.  It is
named to be collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-11, "c64": 2e-5}


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_static_expval_matches_handle_expval_twice(dtype):
    import paper_2508_13615_gb300 as L
    from paper_2508_13615_gb300 import lqs as B
    n = 14
    terms = W.tfim(n) + [W.pauli_word(0.4, {0: "Y", 7: "X", 13: "Z"}), W.Pauli(-0.25, (1 << n) - 1, 0b101)]
    with L.StateVector(n, dtype) as sv:
        sv.set_basis(0)
        sv.apply(W.ansatz(n, 2, 12), fused=True)
        e_ref, per_ref = sv.expval(terms)
        ptr, _, code = L.lqs_sv_info(sv.h)
        pa = B.PauliArray(terms)
        lib = ctypes.CDLL(B.LIB_PATH)
        lib.lqs_expval_static.restype = ctypes.c_int
        for _ in range(2):
            out = ctypes.c_double()
            per = np.zeros(len(terms))
            rc = lib.lqs_expval_static(ctypes.c_void_p(ptr), ctypes.c_int(n), ctypes.c_int(code),
                                       ctypes.c_void_p(sv.stream.cuda_stream), pa.ptr(), ctypes.c_int(pa.n),
                                       ctypes.byref(out), per.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
            assert rc == 0, L.lqs_last_error()
            scale = sum(abs(t.coeff) for t in terms)
            assert abs(out.value - e_ref) <= TOL[dtype] * scale
            np.testing.assert_allclose(per, per_ref, atol=TOL[dtype])


def test_static_expval_rejects_too_many_terms():
    import paper_2508_13615_gb300 as L
    n = 8
    with L.StateVector(n, "c128") as sv:
        sv.set_basis(0)
        ptr, _, code = L.lqs_sv_info(sv.h)
        with pytest.raises(L.LqsError) as e:
            L.lqs_expval_static(ptr, n, "c128", [W.pauli_word(1.0, {0: "Z"})] * 65)
        assert e.value.code == L.lqs.LQS_ERR_ARG and "at most 64" in str(e.value)
