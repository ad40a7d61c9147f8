"""The host composition of a gate run into the 32x32 block that goes to the
tensor cores, against the oracle (no GPU): column k of the block is the
oracle's circuit applied to basis state k of five qubits."""
import numpy as np
import pytest

import oracle
import workloads as W

L = pytest.importorskip("paper_2508_13615_gb300")


def oracle_unitary(c):
    cols = [oracle.run_circuit(c, oracle.basis_state(5, k)) for k in range(32)]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_block_matrix_of_random_runs(seed):
    """Every gate of the set (controlled, multi-qubit, user matrices,
    inverses) on five qubits."""
    c = W.random_circuit(5, 80, seed=700 + seed)
    got = L.lqs_block_matrix(c.ops, c.params)
    assert np.max(np.abs(got - oracle_unitary(c))) < 1e-13


def test_block_matrix_of_empty_run_and_errors():
    assert np.array_equal(L.lqs_block_matrix([], np.zeros(0)), np.eye(32))
    c = W.Circuit(6).add("H", (5,))
    with pytest.raises(L.LqsError):
        L.lqs_block_matrix(c.ops, c.params)
