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


# complex64 relative bound per gate: float32 rounds each product and sum to
# 2^-24 relative; a gate's outputs carry a few such roundings, which add up
# like a random walk over the gates applied.  Eight units of 2^-24 per
# sqrt(gate) is generous for that, and far below what a half-precision step
# (2^-11) or a float32 step in complex128 (2^-24 against 2^-46) would leave.
C64_REL_UNIT = 8 * 2.0 ** -24


def c64_rel_bound(gates: int) -> float:
    return C64_REL_UNIT * float(np.sqrt(max(int(gates), 0) + 1))


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_state(got, want, dtype: str, gates: int, what=""):
    """Asserts the parity bars on a whole state and returns max |delta|:
    max |delta amp| <= TOL[dtype]; for complex64 also the relative L2 error
    ||delta|| / ||want|| and max |delta| / max |want| within the float32
    rounding bound of `gates` gates (c64_rel_bound, 4x for the maximum)."""
    err = max_abs(got, want)
    assert err <= TOL[dtype], (what, "max abs", err)
    if dtype == "c64":
        bound = c64_rel_bound(gates)
        rel = rel_l2(got, want)
        assert rel <= bound, (what, "relative L2", rel, bound)
        top = float(np.max(np.abs(np.asarray(want))))
        assert err <= 4 * bound * top, (what, "max abs / max amplitude", err / top, 4 * bound)
    return err
