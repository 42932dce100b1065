"""Dense brute-force Hamiltonians for n <= 12 qubits (oracle layer 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every word is turned into the Kronecker product of its 2x2 single-qubit
matrices (Methods, "Qubit Hamiltonians": H = sum_i c_i W_i); the full 2^n x
2^n matrix is summed and then restricted to the rows and columns of the
subspace.  Basis state index = sum_q b_q 2^q (qubit q is bit q), so the
Kronecker product runs from the highest qubit to qubit 0.
"""
from __future__ import annotations

import numpy as np

# rows = bra (row bit), columns = ket (column bit)
SINGLE = {
    0: np.array([[1, 0], [0, -1]], np.complex128),          # Z
    1: np.array([[1, 0], [0, 0]], np.complex128),           # 0 = |0><0|
    2: np.array([[0, 0], [0, 1]], np.complex128),           # 1 = |1><1|
    3: np.array([[0, 1], [1, 0]], np.complex128),           # X
    4: np.array([[0, -1j], [1j, 0]], np.complex128),        # Y
    5: np.array([[0, 1], [0, 0]], np.complex128),           # - = |0><1|
    6: np.array([[0, 0], [1, 0]], np.complex128),           # + = |1><0|
}
IDENTITY = np.eye(2, dtype=np.complex128)


def word_matrix(n: int, word) -> np.ndarray:
    """Full 2^n x 2^n matrix of one word [(qubit, code), ...]."""
    factors = [IDENTITY] * n
    for q, c in word:
        factors[q] = SINGLE[int(c)]
    M = np.ones((1, 1), np.complex128)
    for q in range(n - 1, -1, -1):
        M = np.kron(M, factors[q])
    return M


def full_matrix(op) -> np.ndarray:
    n = op.n_qubits
    assert n <= 12
    H = np.zeros((1 << n, 1 << n), np.complex128)
    for coef, word in op.terms():
        H += coef * word_matrix(n, word)
    return H


def restricted(op, keys: np.ndarray) -> np.ndarray:
    """H_S for a sorted subspace ``keys`` ([D, 1] uint64, n <= 12)."""
    idx = np.asarray(keys[:, 0], np.int64)
    H = full_matrix(op)
    return H[np.ix_(idx, idx)]
