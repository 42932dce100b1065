"""The filter/verify scan (QSD_PATH_FILTER_VERIFY) through the C ABI.

Its rows accumulate the same elements in the same group order with the same
operations as the one-pass scan in hash order, so the two must agree bit for
bit, in every precision mode; both must match the oracle (1e-12 FP64, 2^-22
FP32 storage), for single columns and blocks of 16.  Cases: one- and
four-word keys, spin models with constant
elements (Ising: X groups) and with support patterns (XXZ: flip-flop groups
that vanish on aligned pairs), dimensions that leave a ragged last tile, a
subspace smaller than one warp, and more tiles than the persistent grid.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2.0 ** -22
PATH_SCAN_HASH = 5
PATH_FILTER_VERIFY = 8


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


def case(kind):
    if kind == "ising60":
        return wl.ising_heavy_hex(60, seed=9), wl.flip_subspace(60, 30_001, max_flips=8, seed=9)
    if kind == "ising200":
        return wl.ising_heavy_hex(200, seed=4), wl.flip_subspace(200, 50_003, max_flips=20, seed=5)
    if kind == "xxz":
        return wl.xxz_square(6, 6, 0.5, 1.0), wl.xxz_walk_subspace(6, 6, count=40_000, max_len=12, seed=3)
    if kind == "mixed":
        # single-qubit flips (constant elements) and flip-flop bonds (two-qubit
        # supports): the per-group support size is read at run time
        op = wl.ising_heavy_hex(36, seed=3) + wl.xxz_square(6, 6, 0.5, 1.0)
        return op, wl.xxz_walk_subspace(6, 6, count=20_000, max_len=12, seed=4)
    if kind == "tiny":
        return wl.ising_heavy_hex(30, seed=2), wl.flip_subspace(30, 20, max_flips=3, seed=2)
    raise ValueError(kind)


def forced(ctx, h, sub, x, prec, path, k=1):
    if path == PATH_FILTER_VERIFY:
        ctx.set_tuning(1, 5)
    else:
        ctx.set_tuning(1, 1)
        ctx.set_tuning(2, 1)
        ctx.set_tuning(5, 2)
    try:
        assert ctx.product_path(h, sub, prec, k) == path
        y = ctx.apply_H(h, sub, x, precision=prec)
        ctx.synchronize()
        return y.cpu().double().numpy()
    finally:
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.set_tuning(5, 0)


@pytest.mark.parametrize("kind", ["ising60", "ising200", "xxz", "mixed", "tiny"])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 16])
def test_filter_verify_equals_scan_and_oracle(ctx, kind, prec, k):
    import torch
    op, words = case(kind)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    rng = np.random.default_rng(prec + 7 + k)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    if prec == 0:
        xt, tol = to_cuda(ctx, x, torch.float64), FP64_TOL
    else:
        x = x.astype(np.float32).astype(np.float64)
        xt, tol = to_cuda(ctx, x, torch.float32), FP32_TOL
    y8 = forced(ctx, h, sub, xt, prec, PATH_FILTER_VERIFY, k)
    y5 = forced(ctx, h, sub, xt, prec, PATH_SCAN_HASH, k)
    assert np.array_equal(y8, y5)
    assert rel_err(y8, oracle.apply(op, keys, x).real) <= tol


def test_filter_verify_not_offered_outside_its_limits(ctx):
    # scan groups (fermionic ladder terms) and blocks of 4 keep other paths
    h1, eri = wl.chem_integrals(6, seed=1)
    op = wl.molecular_qubit_operator(h1, eri)
    strings = [v for v in range(1 << 6) if bin(v).count("1") == 3]
    words = wl.product_subspace(strings, strings[:7], 6)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(12, words)
    ctx.set_tuning(1, 5)
    try:
        assert ctx.product_path(h, sub, 0, 1) != PATH_FILTER_VERIFY
        op2, words2 = case("ising60")
        h2 = ctx.load_operator(op2)
        sub2 = ctx.build_subspace(60, words2)
        assert ctx.product_path(h2, sub2, 0, 1) == PATH_FILTER_VERIFY
        assert ctx.product_path(h2, sub2, 0, 16) == PATH_FILTER_VERIFY
        assert ctx.product_path(h2, sub2, 0, 4) != PATH_FILTER_VERIFY
    finally:
        ctx.set_tuning(1, 0)
