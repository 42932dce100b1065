"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each check ties one oracle layer to the paper or to mathematics: the printed
merging table (Tbl. S1), the structural properties of words (Methods,
properties 1-3 and the 1/2^m rule), dense Kronecker products, second
quantisation, Hermiticity, closed-form ground energies and library eigen
solvers.  All run on the CPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import brute, fermion

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _sorted_keys(words):
    return oracle.sort_unique(words)


# ------------------------------------------------------- Tbl. S1 (paper) --
def test_merge_rules_match_table_s1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "merge_rules_tbl_s1.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 16
    for a, b, res in rows:
        assert wl.merge_pair(a, b) == res, (a, b, res)


# ------------------------------------------- Methods, properties 1-3, 1/2^m --
@pytest.mark.parametrize("seed", range(6))
def test_pauli_word_properties(seed):
    rng = np.random.default_rng(seed)
    n = 7
    F_of = {}
    for _ in range(8):
        qs = rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False)
        word = [(int(q), int(rng.choice([wl.Z, wl.X, wl.Y]))) for q in qs]
        M = brute.word_matrix(n, word)
        nz = np.abs(M) > 0
        # property 1: exactly one nonzero per row (and per column)
        assert np.all(nz.sum(axis=1) == 1) and np.all(nz.sum(axis=0) == 1)
        # property 2: column = row XOR (bits under X / Y)
        f = sum(1 << q for q, c in word if c in (wl.X, wl.Y))
        rows, cols = np.nonzero(nz)
        assert np.all(cols == (rows ^ f))
        F_of.setdefault(f, []).append(nz)
    # property 3: words with the same off-diagonal structure share positions
    for f, mats in F_of.items():
        for m in mats[1:]:
            assert np.array_equal(m, mats[0])


@pytest.mark.parametrize("seed", range(6))
def test_projector_ladder_fraction(seed):
    rng = np.random.default_rng(100 + seed)
    n = 8
    qs = rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False)
    word = [(int(q), int(rng.integers(0, 7))) for q in qs]
    m = sum(1 for _, c in word if c in (wl.P0, wl.P1, wl.LOWER, wl.RAISE))
    M = brute.word_matrix(n, word)
    nonzero_rows = int(np.count_nonzero(np.abs(M).sum(axis=1)))
    assert nonzero_rows * (1 << m) == (1 << n)


# ----------------------------------------------- oracle vs dense Kronecker --
@pytest.mark.parametrize("n,T,D,k,seed", [(5, 12, 20, 1, 0), (8, 30, 150, 3, 1),
                                          (10, 40, 400, 2, 2), (6, 25, 64, 1, 3)])
def test_oracle_apply_matches_kronecker(n, T, D, k, seed):
    op = wl.random_extended(n, T, max_weight=n, seed=seed, hermitian=False, real=False)
    keys = _sorted_keys(wl.random_subspace(n, D, seed + 10, duplicates=5))
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(keys.shape[0], k)) + 1j * rng.normal(size=(keys.shape[0], k))
    H = brute.restricted(op, keys)
    assert _rel(oracle.apply(op, keys, x), H @ x) < 1e-13
    assert _rel(oracle.diagonal(op, keys), np.diag(H)) < 1e-13 or np.allclose(np.diag(H), 0)
    assert np.allclose(oracle.dense(op, keys), H, atol=1e-13)


@pytest.mark.parametrize("n,T,D,k,seed", [(6, 20, 50, 1, 20), (9, 35, 300, 4, 21), (12, 30, 900, 2, 22)])
def test_oracle_apply_rows_matches_kronecker_and_apply(n, T, D, k, seed):
    """The sampled-row product (the CPU baseline and the full-size parity
    checker) against dense Kronecker rows and the whole-vector product: rows
    in random order with repeats, k columns, complex non-Hermitian
    coefficients, real x."""
    op = wl.random_extended(n, T, max_weight=n, seed=seed, hermitian=False, real=False)
    keys = _sorted_keys(wl.random_subspace(n, D, seed + 3, duplicates=7))
    Dk = keys.shape[0]
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(Dk, k))
    rows = rng.integers(0, Dk, size=min(Dk, 60))
    rows[-1] = rows[0]  # a repeated row
    H = brute.restricted(op, keys)
    got = oracle.apply_rows(op, keys, x, rows)
    assert got.shape == (rows.shape[0], k)
    assert _rel(got, (H @ x)[rows]) < 1e-13
    assert _rel(got, oracle.apply(op, keys, x)[rows]) < 1e-15
    # one-dimensional x gives one-dimensional rows
    y1 = oracle.apply_rows(op, keys, x[:, 0], rows)
    assert y1.shape == rows.shape and _rel(y1, (H @ x[:, 0])[rows]) < 1e-13


def test_oracle_apply_rows_column_not_row_index():
    """A column's x is read at the column's index: with x = e_c only the rows
    that reach column c see a nonzero, equal to H[row, c]."""
    n = 8
    op = wl.random_extended(n, 24, max_weight=4, seed=31, hermitian=True, real=True)
    keys = _sorted_keys(wl.random_subspace(n, 200, 32))
    Dk = keys.shape[0]
    H = brute.restricted(op, keys)
    rows = np.arange(Dk)
    for c in (0, Dk // 3, Dk - 1):
        x = np.zeros(Dk)
        x[c] = 1.0
        assert np.array_equal(oracle.apply_rows(op, keys, x, rows), H[:, c])


def test_oracle_apply_rows_rejects_complex_x_and_bad_rows():
    op = wl.tfim_chain(6, g=1.0)
    keys = _sorted_keys(wl.full_space(6))
    with pytest.raises(TypeError):
        oracle.apply_rows(op, keys, np.ones(64) * 1j, [0, 1])
    with pytest.raises(oracle.OracleError):
        oracle.apply_rows(op, keys, np.ones(64), [64])


def test_oracle_identity_term_and_empty_subspace():
    op = wl.QubitOperator.from_terms(3, [(2.5, []), (1.0, [(0, "X")])])
    keys = _sorted_keys(wl.full_space(3))
    x = np.arange(8, dtype=float)
    H = brute.restricted(op, keys)
    assert _rel(oracle.apply(op, keys, x), H @ x) < 1e-15
    empty = np.zeros((0, 1), np.uint64)
    assert oracle.apply(op, empty, np.zeros(0)).shape == (0,)


def test_term_and_target_tables_match_kronecker():
    n = 8
    op = wl.random_extended(n, 20, max_weight=5, seed=7, hermitian=True, real=True)
    keys = _sorted_keys(wl.random_subspace(n, 120, 8))
    D = keys.shape[0]
    rows = keys[:, 0].astype(np.int64)
    pos = {int(r): i for i, r in enumerate(rows)}
    tt = oracle.term_table(op, keys)
    words = list(op.terms())
    factor = {1: 1, 2: 1j, 3: -1, 4: -1j}
    mats = [brute.word_matrix(n, w) for _, w in words]
    for t, M in enumerate(mats):
        for a, r in enumerate(rows):
            nzc = np.nonzero(M[r])[0]
            if tt[a, t] == 0:
                assert nzc.size == 0
            else:
                assert nzc.size == 1 and M[r, nzc[0]] == factor[int(tt[a, t])]
    # groups: distinct nonzero column offsets (row XOR column) of the words
    G = oracle.groups(op)
    fsets = {}
    for t, M in enumerate(mats):
        r_, c_ = np.nonzero(M)
        offs = set((r_ ^ c_).tolist())
        assert len(offs) <= 1
        if offs and offs != {0}:
            fsets.setdefault(offs.pop(), []).append(t)
    expected = sorted(fsets, key=lambda f: (bin(f).count("1"), f))
    assert G[:, 0].tolist() == expected
    tg = oracle.target_table(op, keys)
    for g, f in enumerate(expected):
        for a, r in enumerate(rows):
            hit = [t for t in fsets[f] if np.any(mats[t][r])]
            want = -2 if not hit else pos.get(int(r) ^ f, -1)
            assert tg[a, g] == want


# ------------------------------------------------------------ Hermiticity --
def test_hermitian_csr_invariant():
    n = 9
    op = wl.random_extended(n, 40, max_weight=6, seed=11, hermitian=True, real=False)
    keys = _sorted_keys(wl.random_subspace(n, 300, 12))
    indptr, indices, data = oracle.csr(op, keys)
    D = keys.shape[0]
    entries = {}
    for a in range(D):
        cols = indices[indptr[a]:indptr[a + 1]]
        assert np.all(np.diff(cols) > 0) and a in cols
        for c, v in zip(cols, data[indptr[a]:indptr[a + 1]]):
            entries[(a, int(c))] = v
    for (a, c), v in entries.items():
        assert (c, a) in entries
        assert abs(entries[(c, a)] - np.conj(v)) <= 1e-15 * max(1.0, abs(v))
    rng = np.random.default_rng(0)
    x = rng.normal(size=D) + 1j * rng.normal(size=D)
    y = rng.normal(size=D) + 1j * rng.normal(size=D)
    lhs = np.vdot(x, oracle.apply(op, keys, y))
    rhs = np.vdot(oracle.apply(op, keys, x), y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_zero_coefficient_word_adds_no_structure():
    # H = X_0 + 0 * X_1 on the full 2-qubit space: row 0 (00) reaches 01 only
    op = wl.QubitOperator.from_terms(2, [(1.0, [(0, "X")]), (0.0, [(1, "X")])])
    keys = _sorted_keys(wl.full_space(2))
    indptr, indices, data = oracle.csr(op, keys)
    assert list(indices[indptr[0]:indptr[1]]) == [0, 1]
    assert np.allclose(oracle.dense(op, keys), brute.restricted(op, keys))


def load_msob_example():
    rows = []
    with open(os.path.join(GOLDEN, "msob_example_s3.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            bits, inds, msob, tri = line.split()
            rows.append((int(bits, 2), [int(i) for i in inds.split(",")], int(msob), tri))
    return rows


def test_msob_worked_example():
    # Supplementary, "Most-significant off-diagonal bit": the row bit at the
    # largest flipped index decides the triangle once S is indexed in
    # integer order.  Checked on the oracle's CSR of the two flip groups.
    ex = load_msob_example()
    assert len(ex) == 2
    n = 6
    terms, words = [], []
    for row, inds, msob, tri in ex:
        assert msob == max(inds)
        F = sum(1 << i for i in inds)
        assert (((row >> msob) & 1) == 1) == (tri == "lower")
        assert ((row ^ F) < row) == (tri == "lower")
        terms.append((1.0, [(i, "X") for i in inds]))
        words += [row, row ^ F]
    op = wl.QubitOperator.from_terms(n, terms)
    keys = _sorted_keys(wl.ints_to_words(words, n))
    vals = [int(v) for v in wl.words_to_ints(keys)]
    indptr, indices, data = oracle.csr(op, keys)
    for row, inds, msob, tri in ex:
        a = vals.index(row)
        b = vals.index(row ^ sum(1 << i for i in inds))
        assert b in indices[indptr[a]:indptr[a + 1]]
        assert (b < a) == (tri == "lower")


# ------------------------------------------------- closed forms / solvers --
def tfim_closed_form(N, g):
    """Ground energy of the periodic chain H = -sum ZZ - g sum X, N even:
    -sum_n sqrt(1 + g^2 - 2 g cos(pi (2n+1)/N)) (free-fermion solution)."""
    return -sum(math.sqrt(1 + g * g - 2 * g * math.cos(math.pi * (2 * m + 1) / N)) for m in range(N))


@pytest.mark.parametrize("g", [1.0, 0.5, 2.0])
def test_tfim_closed_form(g):
    op = wl.tfim_chain(12, g=g)
    keys = _sorted_keys(wl.full_space(12))
    e_ref = tfim_closed_form(12, g)
    if g == 1.0:
        assert abs(e_ref + 2.0 / math.sin(math.pi / 24)) < 1e-12
    assert abs(oracle.ground_energy(op, keys) - e_ref) <= 1e-10 * abs(e_ref)
    e, steps = oracle.lanczos(op, keys, m_max=200, tol=1e-14, seed=1)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref)


def test_dense_full_space_small():
    op = wl.xxz_square(3, 3, 0.5, 1.0)
    keys = _sorted_keys(wl.full_space(9))
    e_full = np.linalg.eigvalsh(brute.full_matrix(op).real)[0]
    assert abs(oracle.ground_energy(op, keys) - e_full) < 1e-11
    e, _ = oracle.lanczos(op, keys, m_max=300, tol=1e-14, seed=2)
    assert abs(e - e_full) < 1e-10 * abs(e_full)


def test_lanczos_on_subspace_matches_eigh():
    op = wl.xxz_square(4, 4, 0.5, 1.0)
    keys = _sorted_keys(wl.xxz_walk_subspace(4, 4, count=1500, max_len=8, seed=5))
    H = brute.restricted(op, keys) if op.n_qubits <= 12 else oracle.dense(op, keys)
    e_ref = np.linalg.eigvalsh(H.real)[0]
    e, _ = oracle.lanczos(op, keys, m_max=300, tol=1e-14, seed=3)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref)


def test_tridiag_min_matches_eigvalsh():
    rng = np.random.default_rng(4)
    for m in (1, 2, 7, 60):
        a, b = rng.normal(size=m), rng.normal(size=m)
        T = np.diag(a) + np.diag(b[1:], 1) + np.diag(b[1:], -1)
        assert abs(oracle.tridiag_min(a, b) - np.linalg.eigvalsh(T)[0]) < 1e-13


# ------------------------------------------------------ fermionic layer --
def _random_fermionic(n_modes, n_terms, seed):
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(n_terms):
        L = int(rng.integers(1, 5))
        ops = [(int(rng.integers(0, n_modes)), bool(rng.integers(0, 2))) for _ in range(L)]
        terms.append((complex(rng.normal(), rng.normal()), ops))
    return wl.FermionicOperator(n_modes, terms)


@pytest.mark.parametrize("seed", range(5))
def test_jordan_wigner_matches_second_quantisation(seed):
    fop = _random_fermionic(6, 25, seed)
    qop = wl.jordan_wigner(fop)
    assert set(np.unique(qop.op_code).tolist()) <= {wl.Z, wl.P0, wl.P1, wl.LOWER, wl.RAISE}
    np.testing.assert_allclose(brute.full_matrix(qop), fermion.dense(fop), atol=1e-13)


@pytest.mark.parametrize("n_orb,seed", [(2, 0), (3, 1), (4, 2)])
def test_vectorised_jordan_wigner_matches_second_quantisation(n_orb, seed):
    h1, eri = wl.chem_integrals(n_orb, seed=seed)
    fop = wl.molecular_fermionic(h1, eri)
    qop = wl.molecular_qubit_operator(h1, eri)
    np.testing.assert_allclose(brute.full_matrix(qop), fermion.dense(fop), atol=1e-13)


def test_vectorised_jordan_wigner_two_words_matches_second_quantisation():
    """72 modes (two-word keys): the vectorised transform of a sparse
    molecular operator, restricted to a product subspace, equals the matrix
    that second quantisation gives on the same occupation strings."""
    n_orb = 36
    h1, eri = wl.chem_integrals(n_orb, seed=5)
    eri = np.where(np.abs(eri) >= 0.045, eri, 0.0)
    h1 = np.where(np.abs(h1) >= 0.1, h1, 0.0)
    qop = wl.molecular_qubit_operator(h1, eri)
    fop = wl.molecular_fermionic(h1, eri)
    alpha = wl.excitation_strings(n_orb, 3, 8, 2, 4)
    beta = wl.excitation_strings(n_orb, 3, 7, 2, 1004)
    keys = _sorted_keys(wl.product_subspace(alpha, beta, n_orb))
    assert keys.shape[1] == 2
    states = [int(k[0]) | (int(k[1]) << 64) for k in keys]
    pos = {v: i for i, v in enumerate(states)}
    ref = np.zeros((len(states), len(states)))
    for coef, ops in fop.terms:
        for b, sb in enumerate(states):
            r = fermion.apply_term(ops, sb)
            if r is not None and r[1] in pos:
                ref[pos[r[1]], b] += coef * r[0]
    got = oracle.dense(qop, keys)
    assert np.count_nonzero(np.abs(ref) > 1e-12) > len(states)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_hubbard_dimer_closed_form():
    t, U = 1.0, 3.0
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    op = wl.jordan_wigner(wl.molecular_fermionic(h, eri))
    keys = _sorted_keys(wl.product_subspace([1, 2], [1, 2], 2))
    e = oracle.ground_energy(op, keys)
    assert abs(e - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_one_body_slater_closed_form():
    rng = np.random.default_rng(9)
    n_orb, na, nb = 4, 2, 1
    A = rng.normal(size=(n_orb, n_orb))
    h = (A + A.T) / 2
    op = wl.jordan_wigner(wl.molecular_fermionic(h, np.zeros((n_orb,) * 4)))
    alpha = [v for v in range(1 << n_orb) if bin(v).count("1") == na]
    beta = [v for v in range(1 << n_orb) if bin(v).count("1") == nb]
    keys = _sorted_keys(wl.product_subspace(alpha, beta, n_orb))
    eps = np.linalg.eigvalsh(h)
    assert abs(oracle.ground_energy(op, keys) - (eps[:na].sum() + eps[:nb].sum())) < 1e-12


# ------------------------------------------------------- bit-string layer --
@pytest.mark.parametrize("n", [36, 64, 130, 200])
def test_sort_unique_and_find(n):
    words = wl.random_subspace(n, 500, n, duplicates=100)
    keys = oracle.sort_unique(words)
    ints = sorted(set(wl.words_to_ints(words)))
    assert wl.words_to_ints(keys) == ints
    probe = np.concatenate([words[:50], wl.random_subspace(n, 50, n + 1)])
    got = oracle.find(keys, probe)
    pos = {v: i for i, v in enumerate(ints)}
    assert got.tolist() == [pos.get(v, -1) for v in wl.words_to_ints(probe)]


def test_operator_errors():
    keys = _sorted_keys(wl.full_space(3))
    bad_repeat = wl.QubitOperator.from_terms(3, [(1.0, [(0, "X"), (0, "Z")])])
    bad_range = wl.QubitOperator.from_terms(3, [(1.0, [(3, "X")])])
    with pytest.raises(oracle.OracleError):
        oracle.apply(bad_repeat, keys, np.zeros(8))
    with pytest.raises(oracle.OracleError):
        oracle.apply(bad_range, keys, np.zeros(8))


# ------------------------------------------------------------------ RAMPS --
def test_row_elements_match_kronecker():
    for seed in range(4):
        n = 7
        op = wl.random_extended(n, 25, max_weight=4, seed=40 + seed, hermitian=False, real=False)
        H = brute.full_matrix(op)
        rng = np.random.default_rng(seed)
        for r in rng.integers(0, 1 << n, size=6):
            cols, els = oracle.row_elements(op, np.array([int(r)], np.uint64))
            got = np.zeros(1 << n, np.complex128)
            got[cols[:, 0].astype(np.int64)] = els
            assert int(r) in set(cols[:, 0].tolist())
            assert np.allclose(got, H[int(r)], atol=1e-13)


def _chain_operator(h, d):
    """Four states 00 -> 01 -> 11 -> 10 (qubit 0 is the low bit) coupled in a
    chain by controlled flips, diagonals d[0..3]: a tridiagonal H."""
    terms = [(h[0], [(0, "X"), (1, "0")]),   # 00 <-> 01
             (h[1], [(1, "X"), (0, "1")]),   # 01 <-> 11
             (h[2], [(0, "X"), (1, "1")])]   # 11 <-> 10
    for bits, e in zip(("00", "01", "11", "10"), d):
        # bits[1] is qubit 0, bits[0] is qubit 1
        terms.append((e, [(0, bits[1]), (1, bits[0])]))
    return wl.QubitOperator.from_terms(2, terms)


def test_ramps_reproduces_equation_s2():
    # Supplementary Eq. S2: starting from row 0 with E = H00, the levels of
    # the recursion are the three printed terms of delta / H00
    from oracle import ramps
    h = (0.3, -0.2, 0.25)
    d = (-5.0, -1.0, 0.5, 2.0)
    op = _chain_operator(h, d)
    H00, H11, H22, H33 = d
    t1 = h[0] ** 2 / (H00 * (H00 - H11))
    t2 = 1.0 / (H00 * (H00 - H11)) * (h[0] ** 2 / (H00 - H11) * h[1] ** 2 / (H00 - H22))
    t3 = (1.0 / (H00 * (H00 - H11) * (H00 - H22))
          * (h[0] ** 2 / (H00 - H11) * h[1] ** 2 / (H00 - H22) * h[2] ** 2 / (H00 - H33)))
    start = np.array([[0b00]], np.uint64)
    keys, levels = ramps.ramps(op, start, H00, 0.0)
    assert [list(lv) for lv in levels[:3]] == [[0b01], [0b11], [0b10]]
    assert levels[0][0b01] == pytest.approx(t1, rel=1e-14)
    assert levels[1][0b11] == pytest.approx(t2, rel=1e-14)
    assert levels[2][0b10] == pytest.approx(t3, rel=1e-14)
    assert keys[:, 0].tolist() == [0, 1, 2, 3]
    # the tolerance cuts the chain after the last level above it
    keys, levels = ramps.ramps(op, start, H00, 0.5 * (abs(t2) + abs(t3)))
    assert keys[:, 0].tolist() == [0b00, 0b01, 0b11]
    keys, _ = ramps.ramps(op, start, H00, 2 * abs(t1))
    assert keys[:, 0].tolist() == [0]


def test_ramps_restricted_and_level_limit():
    from oracle import ramps
    op = _chain_operator((0.3, -0.2, 0.25), (-5.0, -1.0, 0.5, 2.0))
    start = np.array([[0]], np.uint64)
    keys, _ = ramps.ramps(op, start, -5.0, 0.0, restrict=np.array([[0], [1], [2]], np.uint64))
    assert keys[:, 0].tolist() == [0, 1]  # 11 (= 3) is outside the allowed set, so 10 is never reached
    keys, levels = ramps.ramps(op, start, -5.0, 0.0, max_levels=2)
    assert len(levels) == 2 and keys[:, 0].tolist() == [0, 1, 3]


# ------------------------------------------------------------- trimming --
def test_trim_hand_example():
    # 3 qubits, diagonal -1.0 Z0 - 0.5 Z1 - 0.25 Z2 over the full space: the
    # lowest diagonal is -1.75 (000), the next -1.25 (100): splitting 0.5.
    # Flip groups: X0 (0.3) -> 0.6, X1 (1e-4) -> 2e-4, X0 X2 (0.02 + 0.01 via
    # two words) -> 0.06, X1 X2 with words 0.1 and -0.1 (combined: 0) -> 0.
    from oracle import trim
    terms = [(1.0, [(0, "Z")]), (0.5, [(1, "Z")]), (0.25, [(2, "Z")]),
             (0.3, [(0, "X")]), (1e-4, [(1, "X")]),
             (0.02, [(0, "X"), (2, "X")]), (0.01, [(0, "Y"), (2, "Y")]),
             (0.1, [(1, "X"), (2, "X")]), (-0.1, [(2, "X"), (1, "X")])]
    op = wl.QubitOperator.from_terms(3, [(-c if i < 3 else c, w) for i, (c, w) in enumerate(terms)])
    keys = _sorted_keys(wl.full_space(3))
    kept, idx, split = trim.trim(op, keys, 0.01)
    assert split == 0.5
    assert kept == {(0b001,), (0b101,)}  # 0.6 and 0.06 pass 0.01, 2e-4 and 0 do not
    assert idx == [0, 1, 2, 3, 5, 6]
    kept, idx, _ = trim.trim(op, keys, 0.0)
    assert kept == {(0b001,), (0b010,), (0b101,), (0b110,)}
    kept, idx, _ = trim.trim(op, keys, 2.0)
    assert kept == set() and idx == [0, 1, 2]
