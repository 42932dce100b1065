"""Block LOBPCG with the shifted Jacobi preconditioner against dense
eigendecompositions of the oracle's H_S (numpy eigvalsh, a library routine)
and the TFIM closed form: the k lowest eigenvalues to 1e-10 relative."""
import math

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


def lowest(op, words, k):
    keys = oracle.sort_unique(words)
    return np.linalg.eigvalsh(oracle.dense(op, keys).real)[:k]


def test_lobpcg_tfim_closed_form(ctx):
    op = wl.tfim_chain(12, g=1.0)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(12, wl.full_space(12))
    ev, info = ctx.lobpcg(h, sub, k=1, tol=1e-10)
    e0 = -2.0 / math.sin(math.pi / 24)
    assert info["status"] == "OK"
    assert abs(ev[0] - e0) <= 1e-10 * abs(e0)


def _case(case):
    if case == "xxz":
        return wl.xxz_square(4, 4, 1.0, 0.5), wl.xxz_walk_subspace(4, 4, 2500, seed=7)
    if case == "chem":
        h1, eri = wl.chem_integrals(6, seed=6)
        strings = [v for v in range(64) if bin(v).count("1") == 3]
        return wl.molecular_qubit_operator(h1, eri), wl.product_subspace(strings, strings, 6)
    if case == "ising":
        return wl.ising_heavy_hex(30, seed=2), wl.flip_subspace(30, 2000, max_flips=4, seed=2)
    if case == "ising200":
        return wl.ising_heavy_hex(200, seed=4), wl.flip_subspace(200, 1500, max_flips=20, seed=4)
    return wl.tfim_chain(8, g=0.7), wl.full_space(8)


@pytest.mark.parametrize("case,k,start", [("xxz", 4, 0), ("xxz", 4, 1), ("chem", 3, 0), ("ising", 2, 0),
                                          ("ising200", 4, 1), ("tfim8", 6, 0)])
def test_lobpcg_lowest_eigenvalues_match_dense(ctx, case, k, start):
    import torch
    op, words = _case(case)
    ref = lowest(op, words, k)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    ev, info, vec = ctx.lobpcg(h, sub, k=k, tol=1e-10, want_vectors=True, max_iters=1500, start=start)
    assert info["status"] == "OK", info
    assert np.max(np.abs(ev - ref)) <= 1e-10 * np.max(np.abs(ref))
    ctx.synchronize()
    G = (vec.T @ vec).cpu().numpy()
    assert np.max(np.abs(G - np.eye(k))) <= 1e-10
    hv = ctx.apply_H(h, sub, vec.contiguous())
    ctx.synchronize()
    r = hv - vec * torch.as_tensor(ev, device=vec.device)
    assert float(r.norm(dim=0).max()) <= 1e-8 * float(np.max(np.abs(ev)))


def test_lobpcg_unpreconditioned_reproducible_and_errors(ctx):
    import paper_2603_18731_gb300 as q
    op, words = _case("chem")
    ref = lowest(op, words, 2)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(12, words)
    ev1, i1 = ctx.lobpcg(h, sub, k=2, tol=1e-9, precondition=1, max_iters=2000)
    ev0, i0 = ctx.lobpcg(h, sub, k=2, tol=1e-9, precondition=0, max_iters=2000)
    for ev, info in ((ev1, i1), (ev0, i0)):
        assert info["status"] == "OK"
        assert np.max(np.abs(ev - ref)) <= 1e-10 * np.max(np.abs(ref))
    again, _ = ctx.lobpcg(h, sub, k=2, tol=1e-9, precondition=1, max_iters=2000)
    assert np.array_equal(again, ev1)  # reproducible
    with pytest.raises(q.QsdError):
        ctx.lobpcg(h, sub, k=17)
    nh = ctx.load_operator(wl.random_extended(12, 20, max_weight=3, seed=1, hermitian=False, letters="XZ+-"))
    with pytest.raises(q.QsdError):
        ctx.lobpcg(nh, sub, k=1)
