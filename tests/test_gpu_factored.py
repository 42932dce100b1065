"""The sector-factored product (product subspaces of alpha and beta strings)
against the CPU oracle, through the C ABI.

The subspace build must recognise exactly the subspaces that are the product
of their distinct halves (integer-exact: the half counts equal numpy's), and
the factored product must match the oracle to 1e-12 (FP64) and 2^-22 (FP32
storage) relative max-norm, for one- and two-word keys, k = 1 ... 21 columns
(ragged column blocks), and Lanczos energies to 1e-10.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2.0 ** -22
PATH_FACTORED = 7
PATH_EXCITATION = 2


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


def chem_case(n_orb, n_elec, n_alpha, n_beta, seed, keep=None):
    """Molecular operator of seeded integrals (optionally only the two-body
    integrals of magnitude >= keep) and the product of two excitation lists."""
    h1, eri = wl.chem_integrals(n_orb, seed=seed)
    if keep is not None:
        eri = np.where(np.abs(eri) >= keep, eri, 0.0)
    op = wl.molecular_qubit_operator(h1, eri)
    alpha = wl.excitation_strings(n_orb, n_elec, n_alpha, 4, seed)
    beta = wl.excitation_strings(n_orb, n_elec, n_beta, 4, seed + 1000)
    return op, wl.product_subspace(alpha, beta, n_orb), alpha, beta


def halves(keys, n):
    """Distinct low and high halves (split n // 2) of integer-sorted keys."""
    split = n // 2
    vals = [int(sum(int(w) << (64 * i) for i, w in enumerate(k))) for k in keys]
    lo = {v & ((1 << split) - 1) for v in vals}
    hi = {v >> split for v in vals}
    return len(lo), len(hi)


@pytest.mark.parametrize("n_orb,n_elec,na,nb", [(8, 3, 20, 15), (36, 4, 30, 25)])
def test_product_subspace_is_factored(ctx, n_orb, n_elec, na, nb):
    _, words, _, _ = chem_case(n_orb, n_elec, na, nb, seed=5, keep=0.02)
    n = 2 * n_orb
    keys = oracle.sort_unique(words)
    sub = ctx.build_subspace(n, words)
    f = sub.factored()
    n_a, n_b = halves(keys, n)
    assert n_a * n_b == keys.shape[0]
    assert f == {**f, "is_product": True, "split": n // 2, "n_a": n_a, "n_b": n_b}
    assert f["neighbours"] > 0
    # one row fewer: no longer a product
    sub2 = ctx.build_subspace(n, keys[1:])
    assert sub2.factored()["is_product"] is False
    sub.free()
    sub2.free()


def test_spin_subspace_is_not_factored(ctx):
    words = wl.xxz_walk_subspace(4, 4, count=2000, max_len=8, seed=3)
    sub = ctx.build_subspace(16, words)
    assert sub.factored()["is_product"] is False


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 3, 16, 21])
def test_factored_product_matches_oracle(ctx, prec, k):
    import torch
    import paper_2603_18731_gb300 as q
    op, words, _, _ = chem_case(10, 4, 60, 50, seed=7)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(20, words)
    assert sub.factored()["is_product"]
    assert ctx.product_path(h, sub, prec, k) == PATH_FACTORED
    rng = np.random.default_rng(prec * 100 + k)
    x = rng.normal(size=(sub.dim, k))
    if prec == q.QSD_FP64:
        xt = to_cuda(ctx, x, torch.float64)
        tol = FP64_TOL
    else:
        x = x.astype(np.float32).astype(np.float64)  # the FP32 storage rounding of the input
        xt = to_cuda(ctx, x, torch.float32)
        tol = FP32_TOL
    y = ctx.apply_H(h, sub, xt, precision=prec)
    ctx.synchronize()
    ref = oracle.apply(op, keys, x).real
    assert rel_err(y.cpu().double().numpy(), ref) <= tol


def test_factored_two_word_keys_match_oracle(ctx):
    import torch
    op, words, _, _ = chem_case(36, 4, 30, 25, seed=5, keep=0.02)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(72, words)
    assert sub.W == 2 and sub.factored()["is_product"]
    assert ctx.product_path(h, sub, 0, 4) == PATH_FACTORED
    x = np.random.default_rng(2).normal(size=(sub.dim, 4))
    y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
    ctx.synchronize()
    assert rel_err(y.cpu().numpy(), oracle.apply(op, keys, x).real) <= FP64_TOL


def test_factored_equals_excitation_path(ctx):
    import torch
    op, words, _, _ = chem_case(12, 4, 70, 60, seed=9)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(24, words)
    x = to_cuda(ctx, np.random.default_rng(4).normal(size=(sub.dim, 16)), torch.float64)
    y7 = ctx.apply_H(h, sub, x)
    ctx.set_tuning(1, 2)
    try:
        assert ctx.product_path(h, sub, 0, 16) == PATH_EXCITATION
        y2 = ctx.apply_H(h, sub, x)
    finally:
        ctx.set_tuning(1, 0)
    ctx.synchronize()
    assert rel_err(y7.cpu().numpy(), y2.cpu().numpy()) <= 1e-13
    # a deterministic path: the same call twice gives the same bits
    y7b = ctx.apply_H(h, sub, x)
    ctx.synchronize()
    assert np.array_equal(y7.cpu().numpy(), y7b.cpu().numpy())


@pytest.mark.parametrize("prec", [0, 1])
def test_factored_ground_energy(ctx, prec):
    op, words, _, _ = chem_case(8, 3, 40, 35, seed=11)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(16, words)
    assert ctx.product_path(h, sub, prec, 1) == PATH_FACTORED
    e, info = ctx.lanczos_ground_state(h, sub, precision=prec, max_steps=300, tol=1e-9, check=False)
    e_ref = oracle.ground_energy(op, keys)
    assert abs(e - e_ref) <= (1e-10 if prec == 0 else 1e-7) * abs(e_ref), (e, e_ref, info)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 16])
def test_linear_half_sums_are_bitwise_the_term_sums(ctx, prec, k):
    # the per-pair half-sum tables of the linear ranges (K plus the
    # coefficients of each half string's occupied qubits) give the same
    # fixed-point integers as summing the row's coefficients: bitwise equal
    # products, on a fresh pair (tables off, then built on first use)
    import torch
    import paper_2603_18731_gb300 as q
    op, words, _, _ = chem_case(10, 4, 60, 50, seed=11)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(20, words)
    assert h.info()["n_linear_ranges"] > 0
    rng = np.random.default_rng(3 + k)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    xt = to_cuda(ctx, x, torch.float64 if prec == q.QSD_FP64 else torch.float32)
    ctx.set_tuning(6, 0)
    y_off = ctx.apply_H(h, sub, xt, precision=prec)
    ctx.set_tuning(6, 1)
    y_on = ctx.apply_H(h, sub, xt, precision=prec)
    ctx.synchronize()
    assert torch.equal(y_on, y_off)
    keys = oracle.sort_unique(words)
    xr = x if prec == q.QSD_FP64 else x.astype(np.float32).astype(np.float64)
    tol = FP64_TOL if prec == q.QSD_FP64 else FP32_TOL
    assert rel_err(y_on.cpu().double().numpy(), oracle.apply(op, keys, xr).real) <= tol
    sub.free()
    h.free()
