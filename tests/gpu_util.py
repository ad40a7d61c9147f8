"""Helpers for the GPU parity tests (GPU path through the C ABI vs the oracle)."""
import numpy as np

# Tolerances on max |delta amplitude| (complex128 / complex64), depth <= 200.
TOL = {"c128": 1e-12, "c64": 2e-5}
MODES = [("c128", "df"), ("c128", "f64"), ("c64", "f32")]


def set_mode(arith: str) -> None:
    import paper_2508_13615_gb300 as L
    L.lqs_set_arith({"df": L.LQS_ARITH_DF, "f64": L.LQS_ARITH_F64}.get(arith, L.LQS_ARITH_DF))


def gpu_state(n, dtype, psi0=None, basis=None):
    import paper_2508_13615_gb300 as L
    sv = L.StateVector(n, dtype)
    if psi0 is not None:
        sv.from_numpy(psi0.astype(np.complex64 if dtype == "c64" else np.complex128))
    else:
        sv.set_basis(basis or 0)
    return sv


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - np.asarray(b, dtype=np.complex128))))
