"""GPU RAMPS (Algorithm S1) against the oracle: the output subspace must be
identical as a set of bit-strings (both sides decide |amp| > tau in FP64)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import ramps as oramps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_18731_gb300 as q
    c = q.create(0)
    yield c
    c.close()


def chain_operator(h, d):
    terms = [(h[0], [(0, "X"), (1, "0")]), (h[1], [(1, "X"), (0, "1")]), (h[2], [(0, "X"), (1, "1")])]
    for bits, e in zip(("00", "01", "11", "10"), d):
        terms.append((e, [(0, bits[1]), (1, bits[0])]))
    return wl.QubitOperator.from_terms(2, terms)


def run_both(ctx, op, start, E, tau, max_levels=16, restrict=None):
    h = ctx.load_operator(op)
    s0 = ctx.build_subspace(op.n_qubits, start)
    rs = ctx.build_subspace(op.n_qubits, restrict) if restrict is not None else None
    out, info = ctx.ramps(h, s0, E, tau, max_levels=max_levels, restrict=rs)
    got = ctx.subspace_keys(out)[:out.dim]
    want, levels = oramps.ramps(op, start, E, tau, max_levels=max_levels, restrict=restrict)
    return got, want, info, levels


def test_ramps_chain_equation_s2(ctx):
    op = chain_operator((0.3, -0.2, 0.25), (-5.0, -1.0, 0.5, 2.0))
    got, want, info, levels = run_both(ctx, op, np.array([[0]], np.uint64), -5.0, 0.0)
    assert got[:, 0].tolist() == want[:, 0].tolist() == [0, 1, 2, 3]
    assert info["level_rows"][:3] == [1, 1, 1] and info["rows_out"] == 4
    t2, t3 = abs(levels[1][3]), abs(levels[2][2])
    got, want, info, _ = run_both(ctx, op, np.array([[0]], np.uint64), -5.0, 0.5 * (t2 + t3))
    assert got[:, 0].tolist() == want[:, 0].tolist() == [0, 1, 3]
    got, want, info, _ = run_both(ctx, op, np.array([[0]], np.uint64), -5.0, 0.0, max_levels=2)
    assert got[:, 0].tolist() == [0, 1, 3] and info["stopped_by_limit"] == 1


@pytest.mark.parametrize("n,T,wmax,tau", [(10, 40, 3, 1e-7), (40, 60, 3, 1e-8), (70, 60, 4, 1e-8),
                                          (150, 40, 4, 1e-9)])
def test_ramps_random_operators(ctx, n, T, wmax, tau):
    # weak couplings (0.1 N(0,1)) against Z fields of 3..7 per qubit: the
    # recursion dies out within a few levels
    op = wl.random_extended(n, T, max_weight=wmax, seed=n + T, letters="XYZ01+-")
    op = wl.QubitOperator(op.n_qubits, op.term_ptr, op.op_qubit, op.op_code, op.coef * 0.1)
    op = op + wl.QubitOperator.from_terms(n, [(float(3.0 + q % 5), [(q, "Z")]) for q in range(n)])
    start = wl.random_subspace(n, 3, seed=n)
    keys = oracle.sort_unique(start)
    E = min(float(oracle.diagonal(op, keys)[i].real) for i in range(keys.shape[0])) - 1.0
    got, want, info, _ = run_both(ctx, op, start, E, tau, max_levels=4)
    assert np.array_equal(got, want)
    assert info["rows_out"] == want.shape[0]


def test_ramps_restricted_and_fermionic(ctx):
    h1, eri = wl.chem_integrals(6, seed=6)
    op = wl.molecular_qubit_operator(h1, eri)
    start = wl.ints_to_words([0b000111 | (0b000111 << 6)], 12)  # the HF determinant
    E = float(oracle.diagonal(op, oracle.sort_unique(start))[0].real)
    for tau in (1e-3, 1e-4):
        got, want, info, _ = run_both(ctx, op, start, E, tau, max_levels=3)
        assert np.array_equal(got, want)
    strings = [v for v in range(64) if bin(v).count("1") == 3]
    full = oracle.sort_unique(wl.product_subspace(strings, strings, 6))
    allowed = np.concatenate([full[::3], start])
    got, want, info, _ = run_both(ctx, op, start, E, 1e-4, max_levels=3, restrict=allowed)
    assert np.array_equal(got, want)
