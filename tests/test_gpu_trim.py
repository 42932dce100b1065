"""Operator group trimming on the device against the oracle: the kept flip
sets must be identical, the trimmed operator's product must equal the oracle
product of the kept input words, and the counts must agree."""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import trim as otrim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_18731_gb300 as q
    c = q.create(0)
    yield c
    c.close()


def _scaled_random(n, T, seed):
    # coefficients spread over six decades, so a tolerance cuts between groups
    op = wl.random_extended(n, T, max_weight=3, seed=seed)
    rng = np.random.default_rng(seed)
    scale = 10.0 ** rng.uniform(-6, 0, size=op.n_terms // 2)
    scale = np.concatenate([scale, scale])  # the appended adjoints keep their partners' scale
    op = wl.QubitOperator(op.n_qubits, op.term_ptr, op.op_qubit, op.op_code, op.coef * scale)
    return op + wl.QubitOperator.from_terms(n, [(float(1.0 + 0.37 * q), [(q, "Z")]) for q in range(n)])


@pytest.mark.parametrize("n,T,count,tol", [(10, 60, 600, 1e-3), (70, 80, 2000, 1e-4), (150, 50, 1500, 1e-5)])
def test_trim_matches_oracle(ctx, n, T, count, tol):
    import torch
    op = _scaled_random(n, T, seed=n)
    words = wl.random_subspace(n, count, seed=n)
    keys = oracle.sort_unique(words)
    kept, idx, split = otrim.trim(op, keys, tol)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    t, info = ctx.trim_operator(h, sub, tol)
    got = {tuple(int(v) for v in row) for row in t.groups()[:t.info()["n_groups"]]}
    assert got == kept
    assert info["groups_kept"] == len(kept) and info["terms_kept"] == len(idx)
    assert info["splitting"] == pytest.approx(split, rel=1e-14, abs=0.0)
    all_terms = list(op.terms())
    sub_op = wl.QubitOperator.from_terms(n, [all_terms[i] for i in idx])
    x = np.random.default_rng(1).normal(size=sub.dim)
    ref = oracle.apply(sub_op, keys, x).real
    with torch.cuda.stream(ctx.stream):
        xt = torch.as_tensor(x, device=ctx.device)
    y = ctx.apply_H(t, sub, xt)
    ctx.synchronize()
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_trim_keeps_everything_at_zero_tol_and_chemistry(ctx):
    h1, eri = wl.chem_integrals(6, seed=6)
    op = wl.molecular_qubit_operator(h1, eri)
    strings = [v for v in range(64) if bin(v).count("1") == 3]
    words = wl.product_subspace(strings, strings, 6)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(12, words)
    t0, i0 = ctx.trim_operator(h, sub, 0.0)
    assert i0["groups_kept"] == h.info()["n_groups"]
    for tol in (1e-4, 1e-2):
        kept, idx, split = otrim.trim(op, keys, tol)
        t, info = ctx.trim_operator(h, sub, tol)
        got = {tuple(int(v) for v in row) for row in t.groups()[:t.info()["n_groups"]]}
        assert got == kept and info["terms_kept"] == len(idx)
