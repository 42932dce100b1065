"""Oracle of operator group trimming (Results, chemistry: groups whose matrix
elements are small against the smallest diagonal energy splitting of the
subspace are removed before matrix evaluation).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain Python over the
input words.  Readings: a group is the set of words with one flip set F (the
qubits carrying X, Y, - or +); its elements are bounded by the sum over its
words of |c| (equal words combined first; the (-i)^{#Y} factor has modulus
one); the splitting is the smallest d_r - d_min over the subspace rows with
d_r > d_min; a group is kept when bound / splitting >= tol; diagonal words
(F empty) and the identity are always kept, and every group is kept when
all diagonal entries are equal.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np

from . import diagonal

FLIPS = {3, 4, 5, 6}  # X, Y, -, +


def trim(op, keys: np.ndarray, tol: float):
    """(kept flip sets as a set of int tuples [W words], kept input term
    indices, splitting)."""
    W = keys.shape[1]
    d = diagonal(op, keys).real
    dmin = float(d.min()) if d.size else 0.0
    above = d[d > dmin] - dmin
    split = float(above.min()) if above.size else 0.0
    words = OrderedDict()  # canonical word -> (flip set, summed coefficient)
    flips_of = []
    for t in range(op.n_terms):
        a, b = int(op.term_ptr[t]), int(op.term_ptr[t + 1])
        word = tuple(sorted(zip(op.op_qubit[a:b].tolist(), op.op_code[a:b].tolist())))
        F = [0] * W
        for q, c in word:
            if c in FLIPS:
                F[q >> 6] |= 1 << (q & 63)
        F = tuple(F)
        flips_of.append(F)
        c = complex(op.coef[t])
        if c == 0:
            continue
        f0, s = words.get(word, (F, 0j))
        words[word] = (F, s + c)
    bound = {}
    for F, s in words.values():
        if any(F):
            bound[F] = bound.get(F, 0.0) + abs(s)
    kept = {F for F, m in bound.items() if split == 0.0 or m / split >= tol}
    terms = [t for t in range(op.n_terms) if not any(flips_of[t]) or flips_of[t] in kept]
    return kept, terms, split
