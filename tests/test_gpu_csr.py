"""GPU CSR build (two passes, MSOB lower triangle) against the CPU oracle.

Structure (indptr, indices) must be bit-exact; values within 1e-12 of the
largest entry (FP64 sums of the same terms in another order: the mirrored
upper entries are summed at the row that evaluated them).
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

VAL_TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_18731_gb300 as q
    c = q.create(0)
    yield c
    c.close()


def check_csr(got, ref, complex_data=False):
    indptr, indices, data = got[:3]
    r_ptr, r_ind, r_dat = ref
    assert np.array_equal(indptr.cpu().numpy(), r_ptr)
    assert np.array_equal(indices.cpu().numpy().astype(np.int64), r_ind)
    scale = max(float(np.max(np.abs(r_dat))) if r_dat.size else 0.0, 1e-300)
    assert float(np.max(np.abs(data.cpu().numpy() - r_dat.real), initial=0.0)) <= VAL_TOL * scale
    if complex_data:
        assert float(np.max(np.abs(got[3].cpu().numpy() - r_dat.imag), initial=0.0)) <= VAL_TOL * scale


@pytest.mark.parametrize("n,T,wmax,count", [(10, 40, 4, 700), (70, 60, 5, 3000), (140, 50, 6, 2500),
                                            (300, 30, 4, 1500)])
@pytest.mark.parametrize("full", [False, True])
def test_csr_random_hermitian(ctx, n, T, wmax, count, full):
    op = wl.random_extended(n, T, max_weight=wmax, seed=n + T)
    words = wl.random_subspace(n, count, seed=n)
    # add every single-group neighbour of a few rows so that lookups hit
    keys0 = oracle.sort_unique(words)
    extra = [keys0[:50] ^ f for f in oracle.groups(op)[:20]]
    words = np.concatenate([words] + extra)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    got = ctx.to_csr(h, sub, full=full, index_bits=32 if n < 200 else 64)
    check_csr(got, oracle.csr(op, keys))


def test_csr_spin_and_fermion_models(ctx):
    cases = []
    op = wl.xxz_square(4, 4, 1.0, 0.5)
    cases.append((op, wl.xxz_walk_subspace(4, 4, 3000, seed=2)))
    cases.append((wl.tfim_chain(12), wl.full_space(12)))
    h1, eri = wl.chem_integrals(6, seed=6)
    strings = [v for v in range(1 << 6) if bin(v).count("1") == 3]
    cases.append((wl.molecular_qubit_operator(h1, eri), wl.product_subspace(strings, strings, 6)))
    for op, words in cases:
        keys = oracle.sort_unique(words)
        h = ctx.load_operator(op)
        sub = ctx.build_subspace(op.n_qubits, words)
        ref = oracle.csr(op, keys)
        for full in (False, True):
            check_csr(ctx.to_csr(h, sub, full=full), ref)


def test_csr_complex_hermitian(ctx):
    n = 9
    op = wl.random_extended(n, 40, max_weight=6, seed=11, hermitian=True, real=False)
    words = wl.random_subspace(n, 300, 12)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    assert not h.info()["is_real"]
    sub = ctx.build_subspace(n, words)
    check_csr(ctx.to_csr(h, sub, complex_data=True), oracle.csr(op, keys), complex_data=True)


def test_csr_full_non_hermitian_and_errors(ctx):
    import paper_2603_18731_gb300 as q
    n = 12
    op = wl.random_extended(n, 30, max_weight=4, seed=5, hermitian=False, letters="01XZ+-")
    words = wl.random_subspace(n, 1500, seed=6)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    assert not h.info()["is_hermitian"]
    sub = ctx.build_subspace(n, words)
    check_csr(ctx.to_csr(h, sub, full=True), oracle.csr(op, keys))
    with pytest.raises(q.QsdError) as e:
        ctx.to_csr(h, sub, full=False)
    assert e.value.status == "NOT_HERMITIAN"


def test_csr_matches_product_and_lower_count(ctx):
    import torch
    op = wl.ising_heavy_hex(60, seed=4)
    words = wl.flip_subspace(op.n_qubits, 20000, max_flips=4, seed=4)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    indptr, indices, data = ctx.to_csr(h, sub)
    D = sub.dim
    A = torch.sparse_csr_tensor(indptr, indices.to(torch.int64), data, size=(D, D))
    x = torch.randn(D, dtype=torch.float64, device=ctx.device)
    y = ctx.apply_H(h, sub, x)
    ctx.synchronize()
    ya = (A @ x.unsqueeze(1)).squeeze(1)
    assert float((ya - y).abs().max()) <= 1e-12 * float(y.abs().max())
    # symmetric: the strictly lower part has exactly half the off-diagonal entries
    rows = torch.repeat_interleave(torch.arange(D, device=ctx.device), indptr[1:] - indptr[:-1])
    lower = int((indices.to(torch.int64) < rows).sum())
    upper = int((indices.to(torch.int64) > rows).sum())
    assert lower == upper and lower + upper + D == indices.numel()


def test_csr_empty_and_diagonal_only(ctx):
    n = 8
    op = wl.QubitOperator.from_terms(n, [(1.5, [(0, "Z")]), (-0.5, [(3, "1")])])
    words = wl.random_subspace(n, 50, seed=1)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    check_csr(ctx.to_csr(h, sub), oracle.csr(op, keys))
    empty = ctx.build_subspace(n, np.zeros((0, 1), np.uint64))
    indptr, indices, data = ctx.to_csr(h, empty)
    assert indptr.cpu().tolist() == [0] and indices.numel() == 0


def test_csr_rows_longer_than_a_block_sort(ctx):
    # every row of the full 13-qubit space reaches 4100 columns (> 4096):
    # the per-row sorts hand over to the device sort of all entries
    n = 13
    rng = np.random.default_rng(7)
    masks = set()
    while len(masks) < 4100:
        masks.add(int(rng.integers(1, 1 << n)))
    terms = [(float(rng.normal()), [(q, "X") for q in range(n) if (m >> q) & 1]) for m in sorted(masks)]
    op = wl.QubitOperator.from_terms(n, terms)
    words = wl.full_space(n)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    ref = oracle.csr(op, keys)
    for full in (False, True):
        check_csr(ctx.to_csr(h, sub, full=full), ref)
