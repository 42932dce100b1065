"""Seeded synthetic inputs for the subspace Hamiltonian-vector product.

This module only *writes down* inputs: qubit operators as words over the
extended alphabet with coefficients, fermionic operators as products of
creation/annihilation operators, and subspaces as arrays of bit-strings.  It
evaluates no matrix element, builds no table the method uses and performs no
lookup, so the CUDA library and the CPU oracle can both be fed from it without
sharing any of the method's arithmetic.

Conventions (shared by everything that consumes these inputs):

* Letters of the extended alphabet and their integer codes follow the paper's
  mapping [Z, 0, 1, X, Y, -, +] -> [0..6] (Methods, "Qubit Hamiltonians").
  ``0`` = |0><0|, ``1`` = |1><1|, ``+`` = |1><0| (raising), ``-`` = |0><1|.
* A bit-string over ``n`` qubits is ``W = ceil(n/64)`` little-endian uint64
  words: qubit ``q`` is bit ``q % 64`` of word ``q // 64``.  Arrays of
  bit-strings are row-major ``[count, W]``.
* A qubit operator is stored CSR-like: ``term_ptr[T+1]`` (int64), and per
  single-qubit factor ``op_qubit`` (int32) and ``op_code`` (uint8); ``coef`` is
  complex128 ``[T]``.  An empty word is the identity.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------- alphabet --
Z, P0, P1, X, Y, LOWER, RAISE = 0, 1, 2, 3, 4, 5, 6
LETTERS = "Z01XY-+"
CODE = {c: i for i, c in enumerate(LETTERS)}


def n_words(n_qubits: int) -> int:
    """Number of uint64 words of an ``n_qubits`` bit-string."""
    return max(1, (int(n_qubits) + 63) // 64)


# ---------------------------------------------------------------- operators --
@dataclass
class QubitOperator:
    """A linear combination of words over the extended alphabet."""

    n_qubits: int
    term_ptr: np.ndarray  # int64 [T+1]
    op_qubit: np.ndarray  # int32 [nnz]
    op_code: np.ndarray   # uint8 [nnz]
    coef: np.ndarray      # complex128 [T]

    @property
    def n_terms(self) -> int:
        return int(self.coef.shape[0])

    @classmethod
    def from_terms(cls, n_qubits, terms):
        """Build from an iterable of ``(coef, [(qubit, letter), ...])``.

        ``letter`` is a character of ``LETTERS`` or its integer code.  The
        factors of a word are stored sorted by qubit, as the paper stores them.
        """
        ptr = [0]
        qs, cs, coefs = [], [], []
        for coef, word in terms:
            word = sorted(((int(q), CODE[l] if isinstance(l, str) else int(l))
                           for q, l in word), key=lambda t: t[0])
            for q, c in word:
                qs.append(q)
                cs.append(c)
            ptr.append(len(qs))
            coefs.append(complex(coef))
        return cls(int(n_qubits), np.asarray(ptr, np.int64),
                   np.asarray(qs, np.int32), np.asarray(cs, np.uint8),
                   np.asarray(coefs, np.complex128))

    def terms(self):
        """Yield ``(coef, [(qubit, code), ...])`` per term."""
        for t in range(self.n_terms):
            a, b = self.term_ptr[t], self.term_ptr[t + 1]
            yield self.coef[t], list(zip(self.op_qubit[a:b].tolist(),
                                         self.op_code[a:b].tolist()))

    def __add__(self, other: "QubitOperator") -> "QubitOperator":
        assert self.n_qubits == other.n_qubits
        return QubitOperator(
            self.n_qubits,
            np.concatenate([self.term_ptr, other.term_ptr[1:] + self.term_ptr[-1]]),
            np.concatenate([self.op_qubit, other.op_qubit]),
            np.concatenate([self.op_code, other.op_code]),
            np.concatenate([self.coef, other.coef]))

    def adjoint(self) -> "QubitOperator":
        """Hermitian adjoint: swaps + and -, conjugates coefficients."""
        code = self.op_code.copy()
        code[self.op_code == RAISE] = LOWER
        code[self.op_code == LOWER] = RAISE
        return QubitOperator(self.n_qubits, self.term_ptr.copy(),
                             self.op_qubit.copy(), code, np.conj(self.coef))


# ------------------------------------------------------- spin Hamiltonians --
def tfim_chain(n: int, J: float = 1.0, g: float = 1.0, periodic: bool = True):
    """H = -J sum_i Z_i Z_{i+1} - g sum_i X_i on a chain of ``n`` qubits."""
    terms = []
    nb = n if periodic else n - 1
    for i in range(nb):
        terms.append((-J, [(i, "Z"), ((i + 1) % n, "Z")]))
    for i in range(n):
        terms.append((-g, [(i, "X")]))
    return QubitOperator.from_terms(n, terms)


def square_lattice_bonds(Lx: int, Ly: int):
    """Nearest-neighbour bonds of an Lx x Ly periodic square lattice.

    Site (x, y) is qubit ``y*Lx + x``.  Each site contributes its +x and +y
    bond, so there are 2*Lx*Ly bonds (no duplicates for Lx, Ly >= 3).
    """
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            s = y * Lx + x
            bonds.append((s, y * Lx + (x + 1) % Lx))
            bonds.append((s, ((y + 1) % Ly) * Lx + x))
    return bonds


def xxz_square(Lx: int = 6, Ly: int = 6, j_flip: float = 0.5, j_zz: float = 1.0):
    """H = sum_<ij> j_flip (s+_i s-_j + s-_i s+_j) + j_zz Z_i Z_j, periodic."""
    terms = []
    for i, j in square_lattice_bonds(Lx, Ly):
        terms.append((j_flip, [(i, "+"), (j, "-")]))
        terms.append((j_flip, [(i, "-"), (j, "+")]))
        terms.append((j_zz, [(i, "Z"), (j, "Z")]))
    return QubitOperator.from_terms(Lx * Ly, terms)


def xxz_chain_pauli(L: int, J: float = 0.3):
    """The paper's open XXZ chain, H = sum_i J(X_iX_{i+1} + Y_iY_{i+1}) + Z_iZ_{i+1}
    (Results, first equation), written with Pauli letters."""
    terms = []
    for i in range(L - 1):
        terms.append((J, [(i, "X"), (i + 1, "X")]))
        terms.append((J, [(i, "Y"), (i + 1, "Y")]))
        terms.append((1.0, [(i, "Z"), (i + 1, "Z")]))
    return QubitOperator.from_terms(L, terms)


def heavy_hex_graph(n_nodes: int = 200, seed: int = 4, rows: int = 14, cols: int = 28):
    """A heavy-hex-like graph: a brick-wall honeycomb patch with every edge
    subdivided (original vertices have degree <= 3, edge vertices degree 2),
    cut to the first ``n_nodes`` vertices in BFS order from a seeded start and
    relabelled 0..n_nodes-1 in that order.  Returns a list of edges (i < j).
    """
    rng = np.random.default_rng(seed)
    idx = lambda r, c: r * cols + c
    base_edges = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols:
                base_edges.append((idx(r, c), idx(r, c + 1)))
            if r + 1 < rows and (r + c) % 2 == 0:
                base_edges.append((idx(r, c), idx(r + 1, c)))
    nv = rows * cols
    adj = [[] for _ in range(nv + len(base_edges))]
    for e, (a, b) in enumerate(base_edges):
        m = nv + e  # the vertex that subdivides edge e
        adj[a].append(m); adj[m].append(a)
        adj[b].append(m); adj[m].append(b)
    start = int(rng.integers(0, nv))
    order, seen, head = [start], {start}, 0
    while head < len(order) and len(order) < n_nodes:
        v = order[head]; head += 1
        for u in sorted(adj[v]):
            if u not in seen and len(order) < n_nodes:
                seen.add(u); order.append(u)
    if len(order) < n_nodes:
        raise ValueError("patch too small for n_nodes")
    label = {v: i for i, v in enumerate(order)}
    edges = set()
    for v in order:
        for u in adj[v]:
            if u in label:
                a, b = sorted((label[v], label[u]))
                edges.add((a, b))
    return sorted(edges)


def ising_heavy_hex(n_nodes: int = 200, seed: int = 4):
    """H = -sum_<ij> J_ij Z_i Z_j - sum_i h_i X_i on ``heavy_hex_graph`` with
    J_ij ~ U(0.5, 1.5) and h_i ~ U(0.2, 1.0) drawn from ``seed``."""
    edges = heavy_hex_graph(n_nodes, seed)
    rng = np.random.default_rng(seed + 1000)
    J = rng.uniform(0.5, 1.5, size=len(edges))
    h = rng.uniform(0.2, 1.0, size=n_nodes)
    terms = [(-J[e], [(i, "Z"), (j, "Z")]) for e, (i, j) in enumerate(edges)]
    terms += [(-h[i], [(i, "X")]) for i in range(n_nodes)]
    return QubitOperator.from_terms(n_nodes, terms)


def random_extended(n: int, n_terms: int, max_weight: int, seed: int,
                    letters: str = LETTERS, hermitian: bool = True,
                    real: bool = True):
    """Random words over ``letters`` with random coefficients.

    With ``hermitian`` the adjoint of every term is appended, so the sum is
    Hermitian.  With ``real`` the coefficients are chosen so that each matrix
    element is real: a word with an odd number of Y letters gets an imaginary
    coefficient (Y carries a factor of +-i).
    """
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(n_terms):
        w = int(rng.integers(1, max_weight + 1))
        qs = rng.choice(n, size=min(w, n), replace=False)
        word = [(int(q), letters[int(rng.integers(0, len(letters)))]) for q in qs]
        ny = sum(1 for _, l in word if l == "Y")
        c = float(rng.normal())
        if real:
            coef = c * (1j if ny % 2 else 1.0)
        else:
            coef = complex(c, float(rng.normal()))
        terms.append((coef, word))
    op = QubitOperator.from_terms(n, terms)
    if hermitian:
        op = op + op.adjoint()
    return op


# -------------------------------------------------------------- subspaces --
def ints_to_words(values, n_qubits: int) -> np.ndarray:
    """Python ints -> ``[count, W]`` uint64 little-endian words."""
    W = n_words(n_qubits)
    out = np.zeros((len(values), W), np.uint64)
    mask = (1 << 64) - 1
    for i, v in enumerate(values):
        v = int(v)
        for w in range(W):
            out[i, w] = (v >> (64 * w)) & mask
    return out


def words_to_ints(words: np.ndarray):
    """``[count, W]`` uint64 words -> list of Python ints."""
    words = np.asarray(words, np.uint64)
    out = []
    for row in words:
        v = 0
        for w in range(row.shape[0] - 1, -1, -1):
            v = (v << 64) | int(row[w])
        out.append(v)
    return out


def full_space(n: int) -> np.ndarray:
    """Every bit-string of ``n`` <= 24 qubits, in integer order."""
    assert n <= 24
    return np.arange(1 << n, dtype=np.uint64).reshape(-1, 1)


def random_subspace(n: int, count: int, seed: int, duplicates: int = 0) -> np.ndarray:
    """``count`` uniform random bit-strings over ``n`` qubits (not deduplicated),
    with ``duplicates`` extra copies of random earlier rows, shuffled."""
    rng = np.random.default_rng(seed)
    W = n_words(n)
    words = rng.integers(0, 2 ** 63, size=(count, W), dtype=np.uint64) * np.uint64(2) \
        + rng.integers(0, 2, size=(count, W), dtype=np.uint64)
    top = n - 64 * (W - 1)
    if top < 64:
        words[:, W - 1] &= np.uint64((1 << top) - 1)
    if duplicates and count:
        extra = words[rng.integers(0, count, size=duplicates)]
        words = np.concatenate([words, extra])
        words = words[rng.permutation(words.shape[0])]
    return words


def neel_square(Lx: int, Ly: int) -> int:
    """Neel bit-string of the Lx x Ly lattice: site (x, y) set iff (x+y) odd."""
    v = 0
    for y in range(Ly):
        for x in range(Lx):
            if (x + y) % 2:
                v |= 1 << (y * Lx + x)
    return v


def xxz_walk_subspace(Lx: int = 6, Ly: int = 6, count: int = 300_000,
                      max_len: int = 12, seed: int = 2) -> np.ndarray:
    """Distinct bit-strings from random bond-swap walks from the Neel state.

    Each walk starts at the Neel state, draws a length L ~ U{1..max_len}, and L
    times swaps the two bits of a uniformly random lattice bond (a no-op when
    they are equal).  Walks are drawn in seeded batches until ``count``
    distinct strings exist; the first ``count`` distinct strings in the order
    they were produced are returned.  Requires Lx*Ly <= 64.
    """
    n = Lx * Ly
    assert n <= 64
    bonds = np.asarray(square_lattice_bonds(Lx, Ly), np.uint64)
    rng = np.random.default_rng(seed)
    neel = np.uint64(neel_square(Lx, Ly))
    seen: dict[int, None] = {}
    one = np.uint64(1)
    while len(seen) < count:
        batch = max(4096, 2 * (count - len(seen)))
        state = np.full(batch, neel, np.uint64)
        length = rng.integers(1, max_len + 1, size=batch)
        for step in range(max_len):
            b = rng.integers(0, bonds.shape[0], size=batch)
            i, j = bonds[b, 0], bonds[b, 1]
            bi = (state >> i) & one
            bj = (state >> j) & one
            flip = (bi != bj) & (length > step)
            state = np.where(flip, state ^ ((one << i) | (one << j)), state)
        for v in state.tolist():
            if len(seen) >= count:
                break
            seen.setdefault(v, None)
    return np.asarray(list(seen.keys()), np.uint64).reshape(-1, 1)


def flip_subspace(n: int, count: int, max_flips: int = 20, seed: int = 4) -> np.ndarray:
    """Distinct strings, each a seeded uniform reference with d ~ U{1..max_flips}
    distinct uniformly chosen bits flipped; the first ``count`` distinct strings
    in generation order are returned as ``[count, W]`` words."""
    rng = np.random.default_rng(seed)
    W = n_words(n)
    ref = random_subspace(n, 1, seed + 7)[0]
    seen: dict[bytes, None] = {}
    rows = []
    chunk = 65536
    while len(rows) < count:
        d = rng.integers(1, max_flips + 1, size=chunk)
        keys = rng.random((chunk, n), dtype=np.float32)
        pos = np.argpartition(keys, max_flips - 1, axis=1)[:, :max_flips]
        # a uniform random subset of size d: the first d of a random order of the
        # max_flips smallest keys
        sub = np.take_along_axis(keys, pos, axis=1)
        pos = np.take_along_axis(pos, np.argsort(sub, axis=1), axis=1)
        mat = np.tile(ref, (chunk, 1))
        sel = np.arange(max_flips)[None, :] < d[:, None]
        r_idx = np.repeat(np.arange(chunk), max_flips)[sel.ravel()]
        q = pos.ravel()[sel.ravel()].astype(np.int64)
        bit = (np.uint64(1) << (q % 64).astype(np.uint64))
        np.bitwise_xor.at(mat, (r_idx, q // 64), bit)
        for row in mat:
            key = row.tobytes()
            if key not in seen:
                seen[key] = None
                rows.append(row.copy())
                if len(rows) >= count:
                    break
    return np.asarray(rows, np.uint64).reshape(count, W)


def flip_words(n: int, count: int, max_flips: int, seed: int, ref=None) -> np.ndarray:
    """``count`` candidate strings (duplicates possible; the library drops
    them), each the reference (seeded uniform unless given) with d ~
    U{1..max_flips} distinct uniformly chosen bits flipped.  The d-subset is
    drawn with Floyd's algorithm, vectorised over rows."""
    rng = np.random.default_rng(seed)
    W = n_words(n)
    ref = random_subspace(n, 1, seed + 7)[0] if ref is None else np.asarray(ref, np.uint64)
    k = min(max_flips, n)
    out = np.empty((count, W), np.uint64)
    chunk = 1 << 17
    for c0 in range(0, count, chunk):
        m = min(chunk, count - c0)
        d = rng.integers(1, k + 1, size=m)
        chosen = np.zeros((m, 64 * W), bool)
        rows = np.arange(m)
        for j in range(n - k, n):
            act = j >= n - d
            t = rng.integers(0, j + 1, size=m)
            pick = np.where(chosen[rows, t], j, t)
            chosen[rows[act], pick[act]] = True
        flips = np.packbits(chosen, axis=1, bitorder="little").view(np.uint64)
        out[c0:c0 + m] = ref[None, :] ^ flips
    return out


def xxz_walk_words(Lx: int, Ly: int, count: int, max_len: int, seed: int) -> np.ndarray:
    """``count`` candidate strings (duplicates possible) from bond-swap walks of
    length U{1..max_len} from the Neel state (as ``xxz_walk_subspace``,
    without dropping duplicates).  Vectorised; Lx*Ly <= 64."""
    bonds = np.asarray(square_lattice_bonds(Lx, Ly), np.uint64)
    rng = np.random.default_rng(seed)
    one = np.uint64(1)
    state = np.full(count, np.uint64(neel_square(Lx, Ly)), np.uint64)
    length = rng.integers(1, max_len + 1, size=count)
    for step in range(max_len):
        b = rng.integers(0, bonds.shape[0], size=count)
        i, j = bonds[b, 0], bonds[b, 1]
        flip = (((state >> i) & one) != ((state >> j) & one)) & (length > step)
        state = np.where(flip, state ^ ((one << i) | (one << j)), state)
    return state.reshape(-1, 1)


# ------------------------------------------------ fermionic Hamiltonians --
@dataclass
class FermionicOperator:
    """Sum of coefficient x ordered product of f^dag (True) / f (False)."""

    n_modes: int
    terms: list  # [(coef, [(mode, is_dagger), ...]), ...]


# Single-mode factors as 2x2 matrices in the basis (|0>, |1>) with rows = bra:
# "+" = |1><0| is the creation operator f^dag, "-" = |0><1| is f.
_MAT = {
    "I": np.eye(2),
    "Z": np.diag([1.0, -1.0]),
    "0": np.array([[1.0, 0.0], [0.0, 0.0]]),
    "1": np.array([[0.0, 0.0], [0.0, 1.0]]),
    "+": np.array([[0.0, 0.0], [1.0, 0.0]]),
    "-": np.array([[0.0, 1.0], [0.0, 0.0]]),
}


def _classify(m):
    """2x2 matrix -> (letter, scale) with m == scale * _MAT[letter]; ('null', 0)
    for the zero matrix."""
    if not np.any(m):
        return "null", 0.0
    for name, b in _MAT.items():
        nz = b != 0
        s = m[nz][0] / b[nz][0]
        if np.allclose(m, s * b, atol=0, rtol=0):
            return name, float(s)
    raise ValueError(f"not a single letter: {m}")


def merge_pair(a: str, b: str) -> str:
    """Product of two single-mode factors over {-, +, 0, 1} written left to
    right as operators act on one fermionic mode (Supplemental Tbl. S1): the
    result is one of the four letters or 'null'.  Every rule of the table has
    scale +1 (the proof is the 2x2 product, done here)."""
    name, s = _classify(_MAT[a] @ _MAT[b])
    if name == "null":
        return "null"
    assert s == 1.0, (a, b, s)
    return name


def jordan_wigner(fop: FermionicOperator) -> QubitOperator:
    """Extended-alphabet Jordan-Wigner transform (Methods, "Fermionic Hamiltonians").

    f_j -> "-" on qubit j with Z on every lower qubit, f^dag_j -> "+" with Z
    on every lower qubit; the ladder operators are not expanded into Paulis.
    The product of a term is formed qubit by qubit: the ordered product of the
    2x2 factors each operator places on a qubit (identity, Z, or its ladder
    letter) is again a scaled single letter of {I, Z, 0, 1, +, -} or zero, so
    the result stays in the extended alphabet.  Equal words are combined by
    summing coefficients and exact zeros are dropped.
    """
    n = fop.n_modes
    acc: dict[tuple, complex] = {}
    for coef, ops in fop.terms:
        scale = complex(coef)
        word = []
        for q in range(n):
            m = np.eye(2)
            for mode, dag in ops:
                if mode == q:
                    m = m @ _MAT["+" if dag else "-"]
                elif mode > q:
                    m = m @ _MAT["Z"]
            name, s = _classify(m)
            if name == "null":
                scale = 0.0
                break
            scale *= s
            if name != "I":
                word.append((q, name))
        if scale == 0:
            continue
        key = tuple(word)
        acc[key] = acc.get(key, 0.0) + scale
    terms = [(c, list(k)) for k, c in acc.items() if c != 0]
    return QubitOperator.from_terms(n, terms)


# ---- vectorised extended-alphabet Jordan-Wigner for molecular Hamiltonians
_MONO = ["I", "Z", "0", "1", "+", "-"]  # single-mode letters; index 6 = null


def _monoid_table():
    """mul[a, b] = (letter of _MAT[a] @ _MAT[b], its scale), null = 6."""
    code = np.zeros((7, 7), np.int8)
    sign = np.zeros((7, 7), np.float64)
    for i, a in enumerate(_MONO):
        for j, b in enumerate(_MONO):
            name, sc = _classify(_MAT[a] @ _MAT[b])
            code[i, j] = 6 if name == "null" else _MONO.index(name)
            sign[i, j] = sc
    code[6, :] = 6
    code[:, 6] = 6
    return code, sign


def jordan_wigner_products(modes: np.ndarray, dags: np.ndarray, coef: np.ndarray, n_modes: int):
    """Extended-alphabet JW of many products of ladder operators at once.

    ``modes``/``dags``: [T, L] mode indices and creation flags of T products of
    L operators (leftmost first); ``coef``: [T].  Same algebra as
    ``jordan_wigner`` (per qubit, the ordered product of the factors each
    operator places there: its ladder letter on its own mode, Z below it), with
    numpy over the T products.  Equal words are combined.  n_modes <= 128.
    """
    assert n_modes <= 128
    code, sign = _monoid_table()
    T, L = modes.shape
    modes = modes.astype(np.int64)
    letter = np.where(dags, 4, 5).astype(np.int8)  # "+" / "-"
    scale = coef.astype(np.float64).copy()
    # product on each touched qubit (one per operator position b); the scale
    # of a qubit touched by several operators is counted once (first position)
    prod = np.zeros((T, L), np.int8)
    for b in range(L):
        qb = modes[:, b]
        p = np.zeros(T, np.int8)  # identity
        acc = np.ones(T)
        for a in range(L):
            f = np.where(modes[:, a] == qb, letter[:, a], np.where(modes[:, a] > qb, 1, 0)).astype(np.int8)
            acc = acc * sign[p, f]
            p = code[p, f]
        prod[:, b] = p
        first = np.ones(T, bool)
        for c in range(b):
            first &= modes[:, c] != qb
        scale = np.where(first, scale * acc, scale)
    # drop null products
    alive = ~np.any(prod == 6, axis=1) & (scale != 0)
    modes, prod, scale = modes[alive], prod[alive], scale[alive]
    T = modes.shape[0]
    NW = (n_modes + 63) // 64
    one = np.uint64(1)
    word = modes // 64
    bits = (one << (modes % 64).astype(np.uint64))  # [T, L] bit within its word
    touched = np.zeros((T, NW), np.uint64)
    zstr = np.zeros((T, NW), np.uint64)
    for a in range(L):
        for w in range(NW):
            on = word[:, a] == w
            touched[:, w] |= np.where(on, bits[:, a], np.uint64(0))
            # Z on every mode below operator a: whole lower words, and the
            # bits below it in its own word
            below = np.where(word[:, a] > w, ~np.uint64(0), np.where(on, bits[:, a] - one, np.uint64(0)))
            zstr[:, w] ^= below
    zstr &= ~touched
    masks = {c: np.zeros((T, NW), np.uint64) for c in range(1, 6)}
    for b in range(L):
        for c in range(1, 6):
            for w in range(NW):
                masks[c][:, w] |= np.where((prod[:, b] == c) & (word[:, b] == w), bits[:, b], np.uint64(0))
    masks[1] |= zstr
    key = np.concatenate([masks[c] for c in range(1, 6)], axis=1)
    # equal words: sort by every key column (the first column most
    # significant), then sum the coefficients of each run
    order = np.lexsort(key.T[::-1])
    ks = key[order]
    start = np.ones(T, bool)
    start[1:] = np.any(ks[1:] != ks[:-1], axis=1)
    run = np.cumsum(start) - 1
    uniq = ks[start]
    csum = np.zeros(uniq.shape[0])
    np.add.at(csum, run, scale[order])
    keep = csum != 0
    uniq, csum = uniq[keep], csum[keep]
    # words: letters on qubits in ascending order
    n = n_modes
    lettermap = {1: Z, 2: P0, 3: P1, 4: RAISE, 5: LOWER}
    mat = np.full((uniq.shape[0], n), 255, np.uint8)
    for c in range(1, 6):
        for w in range(NW):
            col = np.ascontiguousarray(uniq[:, (c - 1) * NW + w]).astype("<u8")
            bitsel = np.unpackbits(col.view(np.uint8).reshape(-1, 8), axis=1, bitorder="little").astype(bool)
            width = min(64, n - 64 * w)
            blk = mat[:, 64 * w:64 * w + width]
            blk[bitsel[:, :width]] = lettermap[c]
    nz = mat != 255
    counts = nz.sum(axis=1)
    term_ptr = np.zeros(uniq.shape[0] + 1, np.int64)
    np.cumsum(counts, out=term_ptr[1:])
    qq = np.nonzero(nz)[1].astype(np.int32)
    cc = mat[nz].astype(np.uint8)
    return QubitOperator(n, term_ptr, qq, cc, csum.astype(np.complex128))


def molecular_qubit_operator(h1: np.ndarray, eri: np.ndarray):
    """The molecular Hamiltonian of ``molecular_fermionic`` (chemists'
    notation, alpha orbital p -> mode p, beta -> n_orb + p) transformed with
    ``jordan_wigner_products`` -- the fast path for larger orbital counts."""
    n = h1.shape[0]
    p, q = np.nonzero(h1)
    m1, d1, c1 = [], [], []
    for s in (0, 1):
        m1.append(np.stack([p + s * n, q + s * n], axis=1))
        d1.append(np.tile([True, False], (p.size, 1)))
        c1.append(h1[p, q])
    P, Q, R, S = np.nonzero(eri)
    v = eri[P, Q, R, S]
    m2, d2, c2 = [], [], []
    for s in (0, 1):
        for t in (0, 1):
            m2.append(np.stack([P + s * n, R + t * n, S + t * n, Q + s * n], axis=1))
            d2.append(np.tile([True, True, False, False], (P.size, 1)))
            c2.append(0.5 * v)
    op1 = jordan_wigner_products(np.concatenate(m1), np.concatenate(d1), np.concatenate(c1), 2 * n)
    op2 = jordan_wigner_products(np.concatenate(m2), np.concatenate(d2), np.concatenate(c2), 2 * n)
    return op1 + op2


def molecular_fermionic(h1: np.ndarray, eri: np.ndarray, const: float = 0.0):
    """H = const + sum_{pq,s} h_pq a+_{ps} a_{qs}
           + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
    in chemists' notation, alpha orbital p -> mode p, beta orbital p -> mode
    n_orb + p.  Zero integrals are skipped."""
    n_orb = h1.shape[0]
    terms = []
    if const:
        terms.append((const, []))
    for s in (0, 1):
        for p in range(n_orb):
            for q in range(n_orb):
                if h1[p, q] != 0:
                    terms.append((h1[p, q], [(p + s * n_orb, True), (q + s * n_orb, False)]))
    for p, q, r, s_ in zip(*(idx.tolist() for idx in np.nonzero(eri))):  # lexicographic (p, q, r, s)
        v = eri[p, q, r, s_]
        for s in (0, 1):
            for t in (0, 1):
                terms.append((0.5 * v, [(p + s * n_orb, True), (r + t * n_orb, True),
                                        (s_ + t * n_orb, False), (q + s * n_orb, False)]))
    return FermionicOperator(2 * n_orb, terms)


def chem_integrals(n_orb: int, seed: int = 3, sigma1: float = 0.1, sigma2: float = 0.05):
    """Seeded one- and two-body integrals: h_pq ~ N(0, sigma1) with h_qp = h_pq,
    and (pq|rs) for each 8-fold-unique index quadruple ~ N(0, sigma2) scaled by
    exp(-|p-q| - |r-s|), expanded by the 8-fold permutational symmetry."""
    rng = np.random.default_rng(seed)
    h = np.zeros((n_orb, n_orb))
    iu = np.triu_indices(n_orb)
    h[iu] = rng.normal(0.0, sigma1, size=iu[0].size)
    h = h + np.triu(h, 1).T
    eri = np.zeros((n_orb,) * 4)
    pairs = [(p, q) for p in range(n_orb) for q in range(p + 1)]
    for a, (p, q) in enumerate(pairs):
        for (r, s) in pairs[: a + 1]:
            v = rng.normal(0.0, sigma2) * math.exp(-abs(p - q) - abs(r - s))
            for (i, j, k, l) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                 (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                eri[i, j, k, l] = v
    return h, eri


def excitation_strings(n_orb: int, n_elec: int, count: int, max_exc: int, seed: int):
    """``count`` distinct n_orb-bit strings of weight ``n_elec``: the
    Hartree-Fock string (lowest n_elec bits) first, then strings made from it by
    e ~ U{1..max_exc} successive random single excitations (a uniformly chosen
    occupied bit moved to a uniformly chosen empty bit)."""
    rng = np.random.default_rng(seed)
    hf = (1 << n_elec) - 1
    seen = {hf: None}
    while len(seen) < count:
        v = hf
        for _ in range(int(rng.integers(1, max_exc + 1))):
            occ = [i for i in range(n_orb) if (v >> i) & 1]
            emp = [i for i in range(n_orb) if not (v >> i) & 1]
            v ^= (1 << occ[int(rng.integers(0, len(occ)))]) | (1 << emp[int(rng.integers(0, len(emp)))])
        seen.setdefault(v, None)
    return list(seen.keys())[:count]


def product_subspace(alpha, beta, n_orb: int) -> np.ndarray:
    """All strings alpha | (beta << n_orb) (beta in the high half), in
    alpha-major order, as ``[len(alpha)*len(beta), W]`` words."""
    n = 2 * n_orb
    if n <= 64:
        a = np.asarray(alpha, np.uint64)
        b = np.asarray(beta, np.uint64) << np.uint64(n_orb)
        return (a[:, None] | b[None, :]).reshape(-1, 1)
    return ints_to_words([a | (b << n_orb) for a in alpha for b in beta], n)
