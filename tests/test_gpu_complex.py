"""Complex product against the oracle (complex FP64 arithmetic from the plain
definition): random complex operators, Hermitian and not, over random
subspaces with one and several word keys; 1e-12 relative max-norm."""
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


@pytest.mark.parametrize("n,T,wmax,count,k,herm", [(9, 50, 6, 400, 1, True), (9, 50, 6, 400, 3, False),
                                                   (70, 80, 5, 3000, 16, True), (130, 60, 4, 2000, 5, False),
                                                   (250, 40, 3, 1500, 1, True)])
def test_complex_product_matches_oracle(ctx, n, T, wmax, count, k, herm):
    import torch
    op = wl.random_extended(n, T, max_weight=wmax, seed=n + k, hermitian=herm, real=False)
    op = op + wl.QubitOperator.from_terms(n, [(0.3 - 0.7j if not herm else 0.3, [])])  # identity term
    words = wl.random_subspace(n, count, seed=n)
    keys0 = oracle.sort_unique(words)
    words = np.concatenate([words] + [keys0[:100] ^ f for f in oracle.groups(op)[:20]])
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    rng = np.random.default_rng(k)
    shape = (sub.dim, k) if k > 1 else (sub.dim,)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    ref = oracle.apply(op, keys, x)
    with torch.cuda.stream(ctx.stream):
        xt = torch.as_tensor(x, device=ctx.device)
    y = ctx.apply_H_complex(h, sub, xt)
    y2 = ctx.apply_H_complex(h, sub, xt)
    ctx.synchronize()
    got = y.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert torch.equal(y, y2)
    if herm:
        # x^H (H y) = (H x)^H y
        yy = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        with torch.cuda.stream(ctx.stream):
            yt = torch.as_tensor(yy, device=ctx.device)
        hy = ctx.apply_H_complex(h, sub, yt)
        ctx.synchronize()
        lhs = np.vdot(x, hy.cpu().numpy())
        rhs = np.vdot(got, yy)
        assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_complex_product_of_real_operator_equals_real_product(ctx):
    import torch
    op = wl.xxz_square(4, 4, 1.0, 0.5)
    words = wl.xxz_walk_subspace(4, 4, 2000, seed=3)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(16, words)
    rng = np.random.default_rng(0)
    xr = rng.normal(size=sub.dim)
    with torch.cuda.stream(ctx.stream):
        xt = torch.as_tensor(xr, device=ctx.device)
        xc = xt.to(torch.complex128)
    y = ctx.apply_H(h, sub, xt)
    yc = ctx.apply_H_complex(h, sub, xc)
    ctx.synchronize()
    assert float((yc.real - y).abs().max()) <= 1e-12 * float(y.abs().max())
    assert float(yc.imag.abs().max()) == 0.0
