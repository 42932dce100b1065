"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Integer results (subspace order and indices, target and term tables) must be
bit-exact.  FP64 products must match to 1e-12 relative max-norm; the FP32
storage path (FP64 accumulation, one rounding per output) to 2^-23 of the
largest output plus the FP32 rounding of the input; ground energies to 1e-10
(FP64) and 1e-7 (FP32-mixed after FP64 refinement) relative.
"""
import math

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
    scale = max(float(np.max(np.abs(b))) if b.size else 0.0, 1e-300)
    return float(np.max(np.abs(a - b))) / scale if a.size else 0.0


def to_cuda(ctx, arr, dtype):
    import torch
    with torch.cuda.stream(ctx.stream):
        return torch.as_tensor(np.ascontiguousarray(arr), device=ctx.device).to(dtype)


def keys_tensor(ctx, words):
    import torch
    with torch.cuda.stream(ctx.stream):
        return torch.as_tensor(np.ascontiguousarray(words).view(np.int64), device=ctx.device)


# ---------------------------------------------------------------- subspace
@pytest.mark.parametrize("n,count,dups", [(12, 3000, 500), (36, 5000, 1000), (64, 4097, 100), (65, 3000, 10),
                                          (130, 2500, 300), (200, 6000, 50), (300, 1500, 20), (20, 1, 0)])
def test_subspace_sorted_keys_and_index_exact(ctx, n, count, dups):
    words = wl.random_subspace(n, count, seed=n + count, duplicates=dups)
    sub = ctx.build_subspace(n, words)
    ref = oracle.sort_unique(words)
    assert sub.dim == ref.shape[0]
    assert np.array_equal(ctx.subspace_keys(sub), ref)
    queries = np.concatenate([words[: min(500, len(words))], wl.random_subspace(n, 300, seed=7 * n)])
    got = ctx.subspace_index(sub, keys_tensor(ctx, queries))
    ctx.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.find(ref, queries))
    sub.free()


def test_subspace_from_device_words_and_empty(ctx):
    words = wl.random_subspace(40, 1000, seed=3, duplicates=100)
    sub = ctx.build_subspace(40, keys_tensor(ctx, words))
    assert np.array_equal(ctx.subspace_keys(sub), oracle.sort_unique(words))
    empty = ctx.build_subspace(40, np.zeros((0, 1), np.uint64))
    assert empty.dim == 0
    got = ctx.subspace_index(empty, keys_tensor(ctx, words[:10]))
    ctx.synchronize()
    assert (got.cpu().numpy() == -1).all()


def test_subspace_rejects_bits_above_n(ctx):
    import paper_2603_18731_gb300 as q
    words = np.array([[1 << 40]], np.uint64)
    with pytest.raises(q.QsdError) as e:
        ctx.build_subspace(36, words)
    assert e.value.status == "QUBIT_RANGE"


# ---------------------------------------------------------------- products
def _check_apply(ctx, op, words, k, seed, mixed=True):
    import torch
    import paper_2603_18731_gb300 as q
    keys = oracle.sort_unique(words)
    D = keys.shape[0]
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(D, k)) if k > 1 else rng.normal(size=D)
    ref = oracle.apply(op, keys, x)
    assert np.max(np.abs(ref.imag)) <= 1e-12 * max(np.max(np.abs(ref.real)), 1.0)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
    ctx.synchronize()
    assert rel_err(y.cpu().numpy(), ref.real) <= FP64_TOL
    if mixed:
        x32 = x.astype(np.float32)
        ref32 = oracle.apply(op, keys, x32.astype(np.float64)).real
        for prec in (q.QSD_FP32_MIXED, q.QSD_FP32_DOT2):
            y32 = ctx.apply_H(h, sub, to_cuda(ctx, x32, torch.float32), precision=prec)
            ctx.synchronize()
            assert rel_err(y32.cpu().numpy().astype(np.float64), ref32) <= FP32_TOL, prec
    return h, sub


@pytest.mark.parametrize("n,T,wmax,count,k", [(10, 40, 6, 700, 1), (36, 60, 8, 3000, 1), (64, 50, 10, 2000, 3),
                                              (70, 50, 8, 2000, 16), (130, 40, 8, 1500, 21), (200, 40, 6, 1200, 4),
                                              (300, 30, 6, 800, 2)])
def test_apply_random_extended_ops(ctx, n, T, wmax, count, k):
    op = wl.random_extended(n, T, max_weight=wmax, seed=n + T, hermitian=True, real=True)
    # subspace closed enough under the operator to give hits: random strings
    # plus their images under random words
    base = wl.random_subspace(n, count // 2, seed=n)
    rng = np.random.default_rng(n)
    ints = wl.words_to_ints(base)
    extra = []
    for v in ints[: count // 2]:
        coef, word = list(op.terms())[int(rng.integers(0, op.n_terms))]
        f = 0
        for qb, c in word:
            if c in (wl.X, wl.Y, wl.LOWER, wl.RAISE):
                f |= 1 << qb
        extra.append(v ^ f)
    words = np.concatenate([base, wl.ints_to_words(extra, n)])
    _check_apply(ctx, op, words, k, seed=n)


def test_apply_tfim_full_space(ctx):
    op = wl.tfim_chain(12, g=1.0)
    _check_apply(ctx, op, wl.full_space(12), 1, seed=1)
    _check_apply(ctx, op, wl.full_space(12), 16, seed=2)


def test_apply_xxz_walk_subspace(ctx):
    op = wl.xxz_square(6, 6)
    words = wl.xxz_walk_subspace(6, 6, count=30_000, seed=2)
    _check_apply(ctx, op, words, 1, seed=3)


def test_apply_fermionic_ladder_groups(ctx):
    n_orb = 4
    h1, eri = wl.chem_integrals(n_orb, seed=5)
    op = wl.jordan_wigner(wl.molecular_fermionic(h1, eri))
    alpha = [v for v in range(1 << n_orb) if bin(v).count("1") == 2]
    words = wl.product_subspace(alpha, alpha, n_orb)
    h, sub = _check_apply(ctx, op, words, 1, seed=4)
    info = h.info()
    assert info["n_ladder_groups"] > 0 and info["is_hermitian"] == 1


def test_apply_deterministic_and_host_path(ctx):
    import torch
    op = wl.xxz_square(4, 4)
    words = wl.xxz_walk_subspace(4, 4, count=5000, seed=1)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(16, words)
    x = np.random.default_rng(0).normal(size=sub.dim)
    xt = to_cuda(ctx, x, torch.float64)
    y1 = ctx.apply_H(h, sub, xt)
    y2 = ctx.apply_H(h, sub, xt)
    ctx.synchronize()
    assert torch.equal(y1, y2)
    yh = ctx.apply_H_host(h, sub, x)
    assert np.array_equal(yh, y1.cpu().numpy())


@pytest.mark.parametrize("n_orb,na,k", [(4, 2, 1), (6, 3, 16), (7, 2, 4)])
def test_excitation_path_matches_scan_and_oracle(ctx, n_orb, na, k):
    import torch
    import paper_2603_18731_gb300 as q
    h1, eri = wl.chem_integrals(n_orb, seed=n_orb)
    op = wl.molecular_qubit_operator(h1, eri)
    strings = [v for v in range(1 << n_orb) if bin(v).count("1") == na]
    words = wl.product_subspace(strings, strings, n_orb)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    info = h.info()
    assert info["n_excitation_groups"] == info["n_groups"] and info["n_excitation_shapes"] == 5
    sub = ctx.build_subspace(op.n_qubits, words)
    rng = np.random.default_rng(n_orb)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    ref = oracle.apply(op, keys, x).real
    x32 = x.astype(np.float32)
    ref32 = oracle.apply(op, keys, x32.astype(np.float64)).real
    outs = {}
    for path in (1, 2):
        ctx.set_tuning(1, path)
        y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
        ctx.synchronize()
        outs[path] = y.cpu().numpy()
        assert rel_err(outs[path], ref) <= FP64_TOL, path
        for prec in (q.QSD_FP32_MIXED, q.QSD_FP32_DOT2):
            y32 = ctx.apply_H(h, sub, to_cuda(ctx, x32, torch.float32), precision=prec)
            ctx.synchronize()
            assert rel_err(y32.cpu().numpy().astype(np.float64), ref32) <= FP32_TOL, (path, prec)
    ctx.set_tuning(1, 0)
    assert rel_err(outs[1], outs[2]) <= FP64_TOL


def test_excitation_rank_index_and_hash_fallback(ctx):
    """Molecular operators find a candidate flip mask's group by its rank (one
    load); an operator whose rank table would be too large (cross-sector
    doubles on 2 x 120 qubits: C(120, 2)^2 > 2^24 entries) keeps the hash
    table.  Both match the oracle."""
    import torch
    h1, eri = wl.chem_integrals(6, seed=6)
    assert ctx.load_operator(wl.molecular_qubit_operator(h1, eri)).info()["excitation_rank_index"] == 1
    n = 240
    rng = np.random.default_rng(12)
    terms = []
    for _ in range(30):
        a, b = (int(v) for v in rng.choice(120, 2, replace=False))
        c, d = (120 + int(v) for v in rng.choice(120, 2, replace=False))
        coef = float(rng.normal())
        terms.append((coef, [(a, "+"), (b, "-"), (c, "+"), (d, "-")]))
        terms.append((coef, [(a, "-"), (b, "+"), (c, "-"), (d, "+")]))
    for _ in range(20):
        off = 120 * int(rng.integers(0, 2))
        a, b = (off + int(v) for v in rng.choice(120, 2, replace=False))
        coef = float(rng.normal())
        terms.append((coef, [(a, "+"), (b, "-")]))
        terms.append((coef, [(a, "-"), (b, "+")]))
    terms.append((0.7, [(3, "Z"), (130, "Z")]))
    op = wl.QubitOperator.from_terms(n, terms)
    words = wl.random_subspace(n, 2000, seed=13)
    keys0 = oracle.sort_unique(words)
    words = np.concatenate([words] + [keys0[:200] ^ f for f in oracle.groups(op)])
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    info = h.info()
    assert info["n_excitation_groups"] > 0 and info["excitation_rank_index"] == 0
    sub = ctx.build_subspace(n, words)
    x = np.random.default_rng(14).normal(size=(sub.dim, 4))
    ref = oracle.apply(op, keys, x).real
    try:
        for path in (1, 2):
            ctx.set_tuning(1, path)
            y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
            ctx.synchronize()
            assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL, path
    finally:
        ctx.set_tuning(1, 0)


def test_excitation_path_with_rest_groups(ctx):
    import torch
    n = 10
    h1, eri = wl.chem_integrals(5, seed=3)
    op = wl.molecular_qubit_operator(h1, eri) + wl.random_extended(n, 15, max_weight=3, seed=4, letters="XYZ")
    words = wl.random_subspace(n, 600, seed=5)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    info = h.info()
    assert 0 < info["n_excitation_groups"] < info["n_groups"]
    sub = ctx.build_subspace(n, words)
    x = np.random.default_rng(1).normal(size=sub.dim)
    ref = oracle.apply(op, keys, x).real
    for path in (1, 2):
        ctx.set_tuning(1, path)
        y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
        ctx.synchronize()
        assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL, path
    ctx.set_tuning(1, 0)


@pytest.mark.parametrize("kind,k", [("chem", 1), ("chem", 16), ("xxz", 1), ("xxz", 4)])
def test_autotuned_product_matches_oracle(ctx, kind, k):
    import torch
    if kind == "chem":
        h1, eri = wl.chem_integrals(8, seed=8)
        op = wl.molecular_qubit_operator(h1, eri)
        strings = [v for v in range(1 << 8) if bin(v).count("1") == 4]
        words = wl.product_subspace(strings, strings, 8)  # 4900 rows
    else:
        op = wl.xxz_square(4, 4, 1.0, 0.5)
        words = wl.xxz_walk_subspace(4, 4, 3000, seed=2)
    keys = oracle.sort_unique(words)
    assert keys.shape[0] >= 2048  # the tuner only measures subspaces this large
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    rng = np.random.default_rng(k)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    ref = oracle.apply(op, keys, x).real
    ctx.set_tuning(3, 0)
    guess = ctx.product_path(h, sub, k=k)
    y0 = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
    ctx.set_tuning(3, 1)
    y1 = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))  # measures, then runs the winner
    tuned = ctx.product_path(h, sub, k=k)
    y2 = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))  # cached choice
    ctx.synchronize()
    if kind == "chem":
        # a product subspace: the factored enumeration, chosen without timing
        assert sub.factored()["is_product"] and guess == tuned == 7
    else:
        assert guess in (0, 1, 2) and tuned in (0, 1, 2, 5)
    for y in (y0, y1, y2):
        assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL
    assert torch.equal(y1, y2)
    ctx.set_tuning(1, {2: 2, 7: 4}.get(tuned, 1))
    if tuned not in (2, 7):
        ctx.set_tuning(2, 8 if tuned == 1 else 1)
        ctx.set_tuning(5, 2 if tuned == 5 else 1)
    assert ctx.product_path(h, sub, k=k) == tuned
    y3 = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
    ctx.synchronize()
    assert torch.equal(y2, y3)  # the cached path is the forced one, bit for bit
    ctx.set_tuning(1, 0)
    ctx.set_tuning(2, 0)
    ctx.set_tuning(5, 0)


@pytest.mark.parametrize("n,T,wmax,count,k,lanes", [(12, 60, 4, 3000, 1, 1), (40, 80, 5, 4000, 4, 8),
                                                     (100, 60, 4, 3000, 16, 1), (250, 40, 3, 2000, 1, 8)])
def test_half_evaluation_matches_oracle(ctx, n, T, wmax, count, k, lanes):
    import torch
    op = wl.random_extended(n, T, max_weight=wmax, seed=n + k)
    words = wl.random_subspace(n, count, seed=n)
    keys0 = oracle.sort_unique(words)
    words = np.concatenate([words] + [keys0[:200] ^ f for f in oracle.groups(op)[:30]])
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    rng = np.random.default_rng(k)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    ref = oracle.apply(op, keys, x).real
    ctx.set_tuning(1, 3)
    ctx.set_tuning(2, lanes)
    assert ctx.product_path(h, sub, k=k) == (4 if lanes == 8 else 3)
    y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
    ctx.synchronize()
    assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL
    # FP32 storage and non-Hermitian operators take the plain scan
    assert ctx.product_path(h, sub, precision=1, k=k) in (0, 1)
    ctx.set_tuning(1, 0)
    ctx.set_tuning(2, 0)


def test_half_evaluation_models_and_tuner(ctx):
    import torch
    cases = [(wl.xxz_square(4, 4, 1.0, 0.5), wl.xxz_walk_subspace(4, 4, 3000, seed=3)),
             (wl.ising_heavy_hex(60, seed=4), wl.flip_subspace(60, 20000, max_flips=3, seed=4))]
    nh = wl.random_extended(10, 30, max_weight=4, seed=5, hermitian=False, letters="01XZ+-")
    for op, words in cases:
        keys = oracle.sort_unique(words)
        h = ctx.load_operator(op)
        sub = ctx.build_subspace(op.n_qubits, words)
        x = np.random.default_rng(2).normal(size=sub.dim)
        ref = oracle.apply(op, keys, x).real
        ctx.set_tuning(4, 1)  # the tuner may pick the half evaluation
        y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
        ctx.synchronize()
        assert ctx.product_path(h, sub) in (0, 1, 3, 4, 5, 6)
        assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL
        ctx.set_tuning(1, 3)
        y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
        ctx.synchronize()
        assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL
        ctx.set_tuning(1, 0)
        ctx.set_tuning(4, 0)
    h = ctx.load_operator(nh)
    sub = ctx.build_subspace(10, wl.random_subspace(10, 500, seed=1))
    ctx.set_tuning(1, 3)
    assert ctx.product_path(h, sub) in (0, 1)
    ctx.set_tuning(1, 0)


# --------------------------------------------------------- integer tables
@pytest.mark.parametrize("n,seed", [(10, 1), (70, 2), (200, 3)])
def test_target_and_term_tables_exact(ctx, n, seed):
    op = wl.random_extended(n, 30, max_weight=5, seed=seed, hermitian=True, real=True)
    base = wl.random_subspace(n, 300, seed=seed)
    ints = wl.words_to_ints(base)
    extra = []
    for i, (coef, word) in enumerate(op.terms()):
        f = sum(1 << qb for qb, c in word if c in (wl.X, wl.Y, wl.LOWER, wl.RAISE))
        extra.append(ints[i % len(ints)] ^ f)
    words = np.concatenate([base, wl.ints_to_words(extra, n)])
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(n, words)
    assert np.array_equal(h.groups(), oracle.groups(op))
    tt = ctx.target_table(h, sub)
    st = ctx.term_table(h, sub)
    ctx.synchronize()
    assert np.array_equal(tt.cpu().numpy(), oracle.target_table(op, keys))
    assert np.array_equal(st.cpu().numpy(), oracle.term_table(op, keys))


def test_diagonal_matches_oracle(ctx):
    op = wl.random_extended(50, 40, max_weight=6, seed=9, hermitian=True, real=True)
    words = wl.random_subspace(50, 2000, seed=9)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(50, words)
    d = ctx.diagonal(h, sub)
    ctx.synchronize()
    assert rel_err(d.cpu().numpy(), oracle.diagonal(op, keys).real) <= FP64_TOL


# ------------------------------------------------------------------ errors
def test_operator_errors(ctx):
    import paper_2603_18731_gb300 as q
    with pytest.raises(q.QsdError) as e:
        ctx.load_operator(wl.QubitOperator.from_terms(3, [(1.0, [(0, "X"), (0, "Z")])]))
    assert e.value.status == "REPEATED_INDEX"
    with pytest.raises(q.QsdError) as e:
        ctx.load_operator(wl.QubitOperator.from_terms(3, [(1.0, [(3, "X")])]))
    assert e.value.status == "QUBIT_RANGE"
    cplx = ctx.load_operator(wl.QubitOperator.from_terms(3, [(1.0, [(0, "Y")])]))
    assert cplx.info()["is_real"] == 0
    sub = ctx.build_subspace(3, wl.full_space(3))
    import torch
    x = to_cuda(ctx, np.ones(8), torch.float64)
    with pytest.raises(q.QsdError) as e:
        ctx.apply_H(cplx, sub, x)
    assert e.value.status == "COMPLEX_UNSUPPORTED"
    nonherm = ctx.load_operator(wl.QubitOperator.from_terms(3, [(1.0, [(0, "+")])]))
    assert nonherm.info()["is_hermitian"] == 0
    with pytest.raises(q.QsdError) as e:
        ctx.lanczos_ground_state(nonherm, sub)
    assert e.value.status == "NOT_HERMITIAN"
    other = ctx.build_subspace(4, wl.full_space(4))
    with pytest.raises(q.QsdError) as e:
        ctx.apply_H(nonherm, other, to_cuda(ctx, np.ones(16), torch.float64))
    assert e.value.status == "INVALID_ARG"


def test_rayleigh_quotient_matches_oracle(ctx):
    import torch
    op = wl.xxz_square(4, 4)
    words = wl.xxz_walk_subspace(4, 4, count=3000, max_len=8, seed=6)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(16, words)
    u = np.random.default_rng(5).normal(size=sub.dim)
    hu = oracle.apply(op, keys, u).real
    theta_ref = float(u @ hu / (u @ u))
    res_ref = float(np.linalg.norm(hu - theta_ref * u) / np.linalg.norm(u))
    theta, res, nrm = ctx.rayleigh_quotient(h, sub, to_cuda(ctx, u, torch.float64))
    assert abs(theta - theta_ref) <= 1e-12 * abs(theta_ref)
    assert abs(res - res_ref) <= 1e-10 * res_ref
    assert abs(nrm - u @ u) <= 1e-12 * (u @ u)


# ------------------------------------------------------------- eigensolver
def test_lanczos_tfim_closed_form(ctx):
    import paper_2603_18731_gb300 as q
    op = wl.tfim_chain(12, g=1.0)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(12, wl.full_space(12))
    e_ref = -2.0 / math.sin(math.pi / 24)
    e, info = ctx.lanczos_ground_state(h, sub, max_steps=200, tol=1e-10)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref), (e, e_ref, info)
    for prec in (q.QSD_FP32_MIXED, q.QSD_FP32_DOT2):
        e2, info2 = ctx.lanczos_ground_state(h, sub, max_steps=200, tol=1e-10, precision=prec)
        assert abs(e2 - e_ref) <= 1e-7 * abs(e_ref), (prec, e2, e_ref, info2)


def test_lanczos_xxz_subspace_vs_oracle(ctx):
    import paper_2603_18731_gb300 as q
    op = wl.xxz_square(4, 4)
    words = wl.xxz_walk_subspace(4, 4, count=2000, max_len=8, seed=5)
    keys = oracle.sort_unique(words)
    e_ref = oracle.ground_energy(op, keys)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(16, words)
    e, info = ctx.lanczos_ground_state(h, sub, max_steps=300, tol=1e-10)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref), (e, e_ref, info)
    for prec in (q.QSD_FP32_MIXED, q.QSD_FP32_DOT2):
        e2, info2 = ctx.lanczos_ground_state(h, sub, max_steps=300, tol=1e-10, precision=prec)
        assert abs(e2 - e_ref) <= 1e-7 * abs(e_ref), (prec, e2, e_ref, info2)


def test_lanczos_hubbard_dimer_closed_form(ctx):
    t, U = 1.0, 3.0
    h1 = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    op = wl.jordan_wigner(wl.molecular_fermionic(h1, eri))
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(4, wl.product_subspace([1, 2], [1, 2], 2))
    e, _ = ctx.lanczos_ground_state(h, sub, max_steps=10, tol=1e-12)
    assert abs(e - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-11


# ------------------------------------------------------------ hash order
def _hash_order_cases():
    h1, eri = wl.chem_integrals(6, seed=9)
    strings = [v for v in range(1 << 6) if bin(v).count("1") == 3]
    return [
        ("xxz", wl.xxz_square(4, 4, 1.0, 0.5), wl.xxz_walk_subspace(4, 4, 3000, seed=5)),
        ("ising200", wl.ising_heavy_hex(200, seed=6), wl.flip_subspace(200, 6000, max_flips=3, seed=6)),
        ("tfim", wl.tfim_chain(12), wl.full_space(12)),
        ("rand70", wl.random_extended(70, 60, max_weight=5, seed=7), wl.random_subspace(70, 3000, seed=7)),
        ("rand140", wl.random_extended(140, 50, max_weight=6, seed=8), wl.random_subspace(140, 2500, seed=8)),
        ("chem", wl.molecular_qubit_operator(h1, eri), wl.product_subspace(strings, strings, 6)),
    ]


@pytest.mark.parametrize("case", range(6))
@pytest.mark.parametrize("k", [1, 4, 16, 21])
def test_hash_order_is_bitwise_index_order(ctx, case, k):
    """Rows taken in bucket order give, row for row, the same bits as rows
    taken by index (same groups in the same order), in every precision; and
    the FP64 result matches the oracle."""
    import torch
    import paper_2603_18731_gb300 as q
    name, op, words = _hash_order_cases()[case]
    keys = oracle.sort_unique(words)
    if name.startswith("rand"):
        words = np.concatenate([words] + [keys[:100] ^ f for f in oracle.groups(op)[:30]])
        keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    rng = np.random.default_rng(k + case)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    ctx.set_tuning(1, 1)
    ctx.set_tuning(2, 1)
    try:
        for prec, dt in ((q.QSD_FP64, torch.float64), (q.QSD_FP32_MIXED, torch.float32),
                         (q.QSD_FP32_DOT2, torch.float32)):
            xd = to_cuda(ctx, x, dt)
            out = {}
            for order in (1, 2):
                ctx.set_tuning(5, order)
                assert ctx.product_path(h, sub, precision=prec, k=k) == (5 if order == 2 else 0)
                out[order] = ctx.apply_H(h, sub, xd, precision=prec)
            ctx.synchronize()
            assert torch.equal(out[1], out[2]), (name, prec)
            if prec == q.QSD_FP64:
                assert rel_err(out[2].cpu().numpy(), oracle.apply(op, keys, x).real) <= FP64_TOL
    finally:
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.set_tuning(5, 0)


@pytest.mark.parametrize("case", [0, 1, 3, 4])
@pytest.mark.parametrize("k", [1, 16])
def test_hash_order_half_evaluation(ctx, case, k):
    import torch
    import paper_2603_18731_gb300 as q
    name, op, words = _hash_order_cases()[case]
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    rng = np.random.default_rng(k)
    x = rng.normal(size=(sub.dim, k)) if k > 1 else rng.normal(size=sub.dim)
    ctx.set_tuning(1, 3)
    ctx.set_tuning(2, 1)
    ctx.set_tuning(5, 2)
    try:
        assert ctx.product_path(h, sub, k=k) == 6
        y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
        ctx.synchronize()
        assert rel_err(y.cpu().numpy(), oracle.apply(op, keys, x).real) <= FP64_TOL
    finally:
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.set_tuning(5, 0)


def test_hash_order_tuner_and_forced_fallbacks(ctx):
    import torch
    import paper_2603_18731_gb300 as q
    op = wl.ising_heavy_hex(60, seed=4)
    words = wl.flip_subspace(60, 20000, max_flips=3, seed=4)
    keys = oracle.sort_unique(words)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(60, words)
    x = np.random.default_rng(3).normal(size=sub.dim)
    ref = oracle.apply(op, keys, x).real
    try:
        ctx.set_tuning(5, 0)
        y = ctx.apply_H(h, sub, to_cuda(ctx, x, torch.float64))
        ctx.synchronize()
        assert ctx.product_path(h, sub) in (0, 1, 5)
        assert rel_err(y.cpu().numpy(), ref) <= FP64_TOL
        # forced hash order keeps 8 lanes per row in index order
        ctx.set_tuning(1, 1)
        ctx.set_tuning(2, 8)
        ctx.set_tuning(5, 2)
        assert ctx.product_path(h, sub) == 1
        # more than 256 qubits: no hash order, the run-time-W scan
        big = wl.random_extended(300, 20, max_weight=3, seed=2)
        hb = ctx.load_operator(big)
        sb = ctx.build_subspace(300, wl.random_subspace(300, 500, seed=2))
        ctx.set_tuning(2, 1)
        assert ctx.product_path(hb, sb) == 0
        with pytest.raises(q.QsdError):
            ctx.set_tuning(5, 3)
    finally:
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.set_tuning(5, 0)
