"""Parity at the benchmark's full sizes, through the C ABI.

The benchmark's workloads are built at their real sizes -- the fermionic
32-orbital operator (1,542,656 terms, 318,928 groups) over 1500 x 1500 alpha
x beta strings (2.25 M rows), the 200-qubit Ising operator over 1 M rows
(four-word keys) and the 6x6 XXZ operator over 300,000 rows -- and the GPU
product, run in the launch configuration the benchmark times, is compared
with the oracle's sampled-row product on rows spread over the whole index
range (first, last and uniformly drawn rows), the XXZ product on every row.
FP64 to 1e-12 and FP32 storage to 2^-22 relative max-norm; the integer
target table bit for bit on sampled row ranges.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2.0 ** -22


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_18731_gb300 as q
    c = q.create(0)
    yield c
    c.close()


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def to_cuda(ctx, arr, dtype):
    import torch
    with torch.cuda.stream(ctx.stream):
        return torch.as_tensor(np.ascontiguousarray(arr), device=ctx.device).to(dtype)


def sample_rows(D, n, seed):
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, 1, D // 2, D - 2, D - 1], rng.choice(D, size=n, replace=False)])
    return np.unique(rows)


def check_rows(ctx, h, sub, op, keys, prec, k, n_rows, seed):
    import torch
    import paper_2603_18731_gb300 as q
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(sub.dim, k))
    if prec == q.QSD_FP64:
        xt, tol = to_cuda(ctx, x, torch.float64), FP64_TOL
    else:
        x = x.astype(np.float32).astype(np.float64)
        xt, tol = to_cuda(ctx, x, torch.float32), FP32_TOL
    y = ctx.apply_H(h, sub, xt, precision=prec)
    ctx.synchronize()
    rows = sample_rows(sub.dim, n_rows, seed + 1)
    got = y[torch.as_tensor(rows, device=y.device)].cpu().double().numpy()
    ref = oracle.apply_rows(op, keys, x, rows).real
    err = rel_err(got, ref)
    assert err <= tol, (prec, k, err)
    return err


# --------------------------------------------- fermionic, 32 orbitals, 2.25 M
@pytest.fixture(scope="module")
def chem(ctx):
    h1, eri = wl.chem_integrals(32, seed=3)
    op = wl.molecular_qubit_operator(h1, eri)
    alpha = wl.excitation_strings(32, 8, 1500, 4, seed=3)
    beta = wl.excitation_strings(32, 8, 1500, 4, seed=1003)
    words = wl.product_subspace(alpha, beta, 32)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(64, words)
    keys = oracle.sort_unique(words)
    yield op, h, sub, keys
    sub.free()
    h.free()


def test_chem_full_size_structure(ctx, chem):
    op, h, sub, keys = chem
    info = h.info()
    assert sub.dim == keys.shape[0] == 2_250_000
    assert info["n_terms_in"] == op.n_terms == 1_542_656
    assert info["n_groups"] == oracle.groups(op).shape[0] == 318_928
    assert info["excitation_rank_index"] == 1
    # the single excitations (2 spins x 496 orbital pairs, two ladder patterns
    # each, four table rows per group) are tabulated as linear ranges
    assert info["n_linear_ranges"] >= 4 * 2 * 496
    f = sub.factored()
    assert f["is_product"] and f["n_a"] == 1500 and f["n_b"] == 1500 and f["split"] == 32
    assert ctx.product_path(h, sub, 0, 16) == 7 and ctx.product_path(h, sub, 1, 16) == 7


def test_chem_full_size_linear_half_sums_bitwise(ctx, chem):
    # 3,968 linear-range rows over 1500 + 1500 half strings: the half-sum
    # tables give bitwise the product that sums each row's coefficients
    import torch
    op, h, sub, keys = chem
    x = np.random.default_rng(5).normal(size=sub.dim)
    with torch.cuda.stream(ctx.stream):
        xt = torch.as_tensor(x, device=ctx.device)
    y_on = ctx.apply_H(h, sub, xt)
    ctx.set_tuning(6, 0)
    y_off = ctx.apply_H(h, sub, xt)
    ctx.set_tuning(6, 1)
    ctx.synchronize()
    assert torch.equal(y_on, y_off)


@pytest.mark.parametrize("prec,k", [(0, 1), (0, 16), (1, 16)])
def test_chem_full_size_sampled_rows(ctx, chem, prec, k):
    op, h, sub, keys = chem
    check_rows(ctx, h, sub, op, keys, prec, k, n_rows=120, seed=30 + 2 * k + prec)


def test_chem_full_size_target_table(ctx, chem):
    op, h, sub, keys = chem
    D = sub.dim
    for r0 in (D // 3, D - 2):
        got = ctx.target_table(h, sub, r0, 2)
        ctx.synchronize()
        ref = oracle.target_table(op, keys, r0, 2)
        assert np.array_equal(got.cpu().numpy(), ref), r0


# ------------------------------------------------- Ising, 200 qubits, 1 M rows
@pytest.fixture(scope="module")
def ising(ctx):
    op = wl.ising_heavy_hex(200, seed=4)
    words = wl.flip_subspace(200, 1_000_000, max_flips=20, seed=4)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(200, words)
    keys = oracle.sort_unique(words)
    yield op, h, sub, keys
    sub.free()
    h.free()


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("prec,k", [(0, 1), (1, 16)])
def test_ising_full_size_sampled_rows(ctx, ising, order, prec, k):
    op, h, sub, keys = ising
    assert sub.dim == 1_000_000
    ctx.set_tuning(5, order)  # index order, hash order
    try:
        check_rows(ctx, h, sub, op, keys, prec, k, n_rows=400, seed=50 + order + 2 * k)
    finally:
        ctx.set_tuning(5, 0)


def test_ising_full_size_target_table(ctx, ising):
    op, h, sub, keys = ising
    D = sub.dim
    for r0 in (0, D // 2, D - 200):
        got = ctx.target_table(h, sub, r0, 200)
        ctx.synchronize()
        assert np.array_equal(got.cpu().numpy(), oracle.target_table(op, keys, r0, 200)), r0


# -------------------------------------------------- XXZ 6x6, 300,000 rows
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_xxz_full_size_every_row(ctx, prec):
    import torch
    import paper_2603_18731_gb300 as q
    op = wl.xxz_square(6, 6, 0.5, 1.0)
    words = wl.xxz_walk_subspace(6, 6, count=300_000, max_len=12, seed=2)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(36, words)
    keys = oracle.sort_unique(words)
    assert sub.dim == 300_000
    x = np.random.default_rng(60 + prec).normal(size=sub.dim)
    if prec == q.QSD_FP64:
        xt, tol = to_cuda(ctx, x, torch.float64), FP64_TOL
    else:
        x = x.astype(np.float32).astype(np.float64)
        xt, tol = to_cuda(ctx, x, torch.float32), FP32_TOL
    y = ctx.apply_H(h, sub, xt, precision=prec)
    ctx.synchronize()
    assert rel_err(y.cpu().double().numpy(), oracle.apply(op, keys, x).real) <= tol
    got = ctx.target_table(h, sub, 150_000, 2000)
    ctx.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.target_table(op, keys, 150_000, 2000))
