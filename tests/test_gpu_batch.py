"""Packed products of many (operator, subspace) pairs from device tile queues.

Each pair's result must equal, bit for bit, the single-pair product on the
path the pack uses for it -- the sector-factored product for a product
subspace with an indexed operator, else the one-lane group scan -- and the
oracle within the FP64 / FP32 parity bounds.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_18731_gb300 as q
    c = q.create(0)
    yield c
    c.close()


def pairs():
    out = [(wl.tfim_chain(10), wl.full_space(10)),
           (wl.xxz_square(4, 4, 1.0, 0.5), wl.xxz_walk_subspace(4, 4, 777, seed=5)),
           (wl.random_extended(70, 40, max_weight=4, seed=1), wl.random_subspace(70, 300, seed=2)),
           (wl.random_extended(12, 30, max_weight=3, seed=3), wl.random_subspace(12, 1, seed=4)),
           (wl.random_extended(12, 30, max_weight=3, seed=3), np.zeros((0, 1), np.uint64)),
           (wl.random_extended(150, 30, max_weight=5, seed=6), wl.random_subspace(150, 513, seed=7)),
           (wl.ising_heavy_hex(60, seed=4), wl.flip_subspace(60, 2600, max_flips=3, seed=8))]
    h1, eri = wl.chem_integrals(4, seed=4)
    strings = [v for v in range(16) if bin(v).count("1") == 2]
    out.append((wl.molecular_qubit_operator(h1, eri), wl.product_subspace(strings, strings, 4)))
    # a factored pair with two-word keys (72 qubits, split 36)
    h1, eri = wl.chem_integrals(36, seed=5)
    eri = np.where(np.abs(eri) >= 0.02, eri, 0.0)
    a = wl.excitation_strings(36, 4, 30, 4, 5)
    b = wl.excitation_strings(36, 4, 25, 4, 1005)
    out.append((wl.molecular_qubit_operator(h1, eri), wl.product_subspace(a, b, 36)))
    return out


@pytest.mark.parametrize("k", [1, 4, 7, 16])
def test_batch_matches_single_and_oracle(ctx, k):
    import torch
    import paper_2603_18731_gb300 as q
    ps = pairs()
    ops = [ctx.load_operator(op) for op, _ in ps]
    subs = [ctx.build_subspace(op.n_qubits, w) for op, w in ps]
    rng = np.random.default_rng(k)
    xs_np = [rng.normal(size=(s.dim, k)) if k > 1 else rng.normal(size=s.dim) for s in subs]
    for prec, tol in ((q.QSD_FP64, 1e-12), (q.QSD_FP32_MIXED, 2.0 ** -22), (q.QSD_FP32_DOT2, 2.0 ** -22)):
        dt = torch.float64 if prec == q.QSD_FP64 else torch.float32
        with torch.cuda.stream(ctx.stream):
            xs = [torch.as_tensor(x, device=ctx.device).to(dt).contiguous() for x in xs_np]
        ys = ctx.apply_H_batch(ops, subs, xs, precision=prec)
        factored = [ctx.product_path(h, s, prec, k) == 7 for h, s in zip(ops, subs)]
        # the fermionic pairs (one- and two-word keys) are product subspaces
        # (so is the one-row subspace of an indexed operator)
        assert factored[-1] and factored[-2] and subs[-1].W == 2
        ctx.set_tuning(1, 1)
        ctx.set_tuning(2, 1)
        singles = [ctx.apply_H(h, s, x, precision=prec) for h, s, x in zip(ops, subs, xs)]
        ctx.set_tuning(1, 4)  # the factored product where it applies
        for i, f in enumerate(factored):
            if f:
                singles[i] = ctx.apply_H(ops[i], subs[i], xs[i], precision=prec)
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.synchronize()
        for (op, words), s, x, y, y1 in zip(ps, subs, xs, ys, singles):
            if s.dim == 0:
                continue
            assert torch.equal(y, y1)
            keys = oracle.sort_unique(words)
            ref = oracle.apply(op, keys, x.double().cpu().numpy()).real
            err = float(np.max(np.abs(y.double().cpu().numpy() - ref)))
            assert err <= tol * max(float(np.max(np.abs(ref))), 1e-300)


def test_batch_errors_and_empty(ctx):
    import torch
    import paper_2603_18731_gb300 as q
    assert ctx.apply_H_batch([], [], []) == []
    op = wl.random_extended(300, 10, max_weight=3, seed=1)
    h = ctx.load_operator(op)
    s = ctx.build_subspace(300, wl.random_subspace(300, 10, seed=1))
    x = torch.zeros(s.dim, dtype=torch.float64, device=ctx.device)
    with pytest.raises(q.QsdError):
        ctx.apply_H_batch([h], [s], [x])  # more than 256 qubits
