"""Oracle of the subspace refinement RAMPS (Supplementary, "Recursive
algorithm for a minimal perturbative subspace", Algorithm S1 and Eq. S2).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain Python over the
C oracle's row enumerator (``row_elements``: every column of a row of H over
the whole Hilbert space with its summed element), for small cases.

The algorithm, in the paper's order: every row of the current level carries a
prefactor (1/E for the starting rows); for every column b_k that the row
reaches through an off-diagonal group, amp = pre |H_jk|^2 / (E - H_kk); a
column with |amp| > tau joins the next level with prefactor amp / (E - H_kk)
and the output subspace; levels repeat until one is empty.

Readings where the printed algorithm is silent or ambiguous:

* A column already in the output (the starting rows or an earlier level) is
  neither added nor expanded again.  Without this the expansion returns to
  its own starting row, where E - H_kk = 0, and the printed expansion Eq. S2
  (a path that never turns back) would not be reproduced.
* The starting rows expand together, level by level (for one starting row,
  the paper's case, this is the printed loop).
* A column reached from several rows of the same level keeps the largest
  |amp| (ties: the larger amp); the printed set/list pair leaves it open.
* A column whose diagonal equals E has an unbounded amp: it is added and not
  expanded.
* ``max_levels`` ends the recursion (the paper's maximum number of
  recursions); ``restrict`` keeps only columns of a given subspace (the
  restricted variant used for the paper's chemistry runs).
"""
from __future__ import annotations

import math

import numpy as np

from . import row_elements


def _key(words: np.ndarray) -> int:
    v = 0
    for w in range(words.shape[0] - 1, -1, -1):
        v = (v << 64) | int(words[w])
    return v


def _words(v: int, W: int) -> np.ndarray:
    return np.array([(v >> (64 * w)) & ((1 << 64) - 1) for w in range(W)], np.uint64)


def diagonal_element(op, v: int, W: int) -> float:
    cols, els = row_elements(op, _words(v, W))
    for c, e in zip(cols, els):
        if _key(c) == v:
            return float(e.real)
    return 0.0


def ramps(op, start_words: np.ndarray, E: float, tau: float, max_levels: int = 16, restrict=None):
    """Returns (sorted output keys [m, W], per-level list of {row: amp})."""
    start_words = np.asarray(start_words, np.uint64)
    W = start_words.shape[1]
    allowed = None if restrict is None else {_key(r) for r in np.asarray(restrict, np.uint64)}
    out = {_key(r) for r in start_words}
    level = {v: 1.0 / E for v in sorted(out)}
    levels = []
    while level and len(levels) < max_levels:
        best = {}  # column -> (amp, E - H_kk)
        for v in sorted(level):
            pre = level[v]
            cols, els = row_elements(op, _words(v, W))
            for c, h in zip(cols, els):
                k = _key(c)
                if k == v or k in out:
                    continue
                if allowed is not None and k not in allowed:
                    continue
                gap = E - diagonal_element(op, k, W)
                amp = math.inf if gap == 0.0 else pre * abs(h) ** 2 / gap
                if not abs(amp) > tau:
                    continue
                old = best.get(k)
                if old is None or abs(amp) > abs(old[0]) or (abs(amp) == abs(old[0]) and amp > old[0]):
                    best[k] = (amp, gap)
        levels.append({k: a for k, (a, _) in best.items()})
        level = {k: (0.0 if g == 0.0 else a / g) for k, (a, g) in best.items()}
        level = {k: p for k, p in level.items() if p != 0.0}
        out.update(best.keys())
    keys = sorted(out)
    return np.array([_words(k, W) for k in keys], np.uint64).reshape(len(keys), W), levels
