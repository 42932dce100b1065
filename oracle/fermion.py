"""Second-quantisation brute force on occupation bit-strings (oracle layer 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Independent of any qubit alphabet: creation and annihilation operators act on
occupation-number states |n_0 n_1 ... >, mode j is bit j, with the canonical
anticommutation sign (-1)^(number of occupied modes below j) (the ordering
that the Jordan-Wigner transform with Z strings on lower modes reproduces,
Methods "Fermionic Hamiltonians").  Used to check the extended-alphabet
Jordan-Wigner input generator on small systems.
"""
from __future__ import annotations

import numpy as np


def apply_term(ops, state: int):
    """Apply the ordered product ``ops`` = [(mode, is_dagger), ...] (leftmost
    acts last) to basis state ``state``.  Returns (sign, new_state) or None."""
    sign = 1
    for mode, dag in reversed(ops):
        occ = (state >> mode) & 1
        if dag == bool(occ):
            return None  # create on occupied / annihilate empty
        below = bin(state & ((1 << mode) - 1)).count("1")
        if below % 2:
            sign = -sign
        state ^= 1 << mode
    return sign, state


def dense(fop) -> np.ndarray:
    """Full 2^n x 2^n matrix of a FermionicOperator, basis index = bits."""
    n = fop.n_modes
    assert n <= 12
    H = np.zeros((1 << n, 1 << n), np.complex128)
    for coef, ops in fop.terms:
        for s in range(1 << n):
            r = apply_term(ops, s)
            if r is not None:
                sign, t = r
                H[t, s] += coef * sign
    return H
