"""GPU tests of the continuous-batching server: requests of different
Hamiltonians and subspace sizes run concurrently and each result equals the
same request solved alone and the oracle's ground energy; admission respects
the memory budget; cancellation and submit-time errors."""
import math
import time

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


def _mix(ctx):
    """(name, operator handle, subspace handle, oracle energy) for a mix of
    families and sizes."""
    cases = []
    op = wl.tfim_chain(12, g=1.0)
    cases.append(("tfim12", op, wl.full_space(12), -2.0 / math.sin(math.pi / 24)))
    for seed, cnt in ((5, 2000), (7, 800)):
        op = wl.xxz_square(4, 4)
        words = wl.xxz_walk_subspace(4, 4, count=cnt, max_len=8, seed=seed)
        cases.append((f"xxz{cnt}", op, words, oracle.ground_energy(op, oracle.sort_unique(words))))
    h1, eri = wl.chem_integrals(4, seed=5)
    op = wl.jordan_wigner(wl.molecular_fermionic(h1, eri))
    alpha = [v for v in range(16) if bin(v).count("1") == 2]
    words = wl.product_subspace(alpha, alpha, 4)
    cases.append(("chem4", op, words, oracle.ground_energy(op, oracle.sort_unique(words))))
    op = wl.ising_heavy_hex(20, seed=3)
    words = wl.flip_subspace(20, 3000, max_flips=6, seed=3)
    cases.append(("ising20", op, words, oracle.ground_energy(op, oracle.sort_unique(words))))
    out = []
    for name, op, words, e in cases:
        out.append((name, ctx.load_operator(op), ctx.build_subspace(op.n_qubits, words), e))
    return out


@pytest.mark.parametrize("precision", [0, 2])
def test_server_mix_equals_alone_and_oracle(ctx, precision):
    import paper_2603_18731_gb300 as q
    cases = _mix(ctx)
    params = dict(precision=precision, max_steps=300, tol=1e-10)
    alone = {}
    for name, h, sub, _ in cases:
        alone[name] = ctx.lanczos_ground_state(h, sub, **params)[0]
    with q.Server(ctx, budget_bytes=1 << 30, max_active=4) as srv:
        tickets = [(name, srv.submit(h, sub, **params), e) for name, h, sub, e in cases for _ in range(2)]
        for name, t, e_ref in tickets:
            r = srv.wait(t, timeout_s=120)
            assert r["status"] == "OK", (name, r)
            tol = 1e-10 if precision == 0 else 1e-7
            assert abs(r["energy"] - e_ref) <= tol * abs(e_ref), (name, r["energy"], e_ref)
            assert abs(r["energy"] - alone[name]) <= 1e-12 * abs(e_ref), (name, r["energy"], alone[name])
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["failed"] == 0


def test_server_budget_and_cancel(ctx):
    import paper_2603_18731_gb300 as q
    cases = _mix(ctx)
    name, h, sub, e_ref = cases[1]  # xxz2000
    with q.Server(ctx, budget_bytes=12 << 20, max_active=8) as srv:
        tickets = [srv.submit(h, sub, max_steps=300, tol=1e-10) for _ in range(6)]
        victim = srv.submit(h, sub, max_steps=300, tol=1e-10)
        srv.cancel(victim)
        for t in tickets:
            r = srv.wait(t, timeout_s=120)
            assert r["status"] == "OK" and abs(r["energy"] - e_ref) <= 1e-10 * abs(e_ref)
        assert srv.wait(victim, timeout_s=120)["status"] in ("CANCELLED", "OK")
        st = srv.stats()
        assert st["peak_bytes"] <= st["budget_bytes"]


def test_server_rejects_bad_requests(ctx):
    import paper_2603_18731_gb300 as q
    nonherm = ctx.load_operator(wl.QubitOperator.from_terms(3, [(1.0, [(0, "+")])]))
    sub = ctx.build_subspace(3, wl.full_space(3))
    with q.Server(ctx, budget_bytes=1 << 28, max_active=2) as srv:
        with pytest.raises(q.QsdError) as e:
            srv.submit(nonherm, sub)
        assert e.value.status == "NOT_HERMITIAN"


@pytest.mark.parametrize("precision", [0, 2])
def test_server_packs_small_requests(ctx, precision):
    # with packing on, every request below 32768 rows joins a pack: its chunks
    # share packed launches with the other members; results equal the
    # request alone
    import paper_2603_18731_gb300 as q
    cases = _mix(ctx)
    params = dict(precision=precision, max_steps=300, tol=1e-10, check_every=10)
    alone = {name: ctx.lanczos_ground_state(h, sub, **params)[0] for name, h, sub, _ in cases}
    for rows in (32768, 0):
        with q.Server(ctx, budget_bytes=1 << 30, max_active=16) as srv:
            srv.set_pack_rows(rows)
            tickets = [(name, srv.submit(h, sub, **params), e) for name, h, sub, e in cases for _ in range(3)]
            steps = 0
            for name, t, e_ref in tickets:
                r = srv.wait(t, timeout_s=120)
                assert r["status"] == "OK", (name, r)
                tol = 1e-10 if precision == 0 else 1e-7
                assert abs(r["energy"] - e_ref) <= tol * abs(e_ref), (name, r["energy"], e_ref)
                assert abs(r["energy"] - alone[name]) <= 1e-12 * abs(e_ref), (name, r["energy"], alone[name])
                steps += r["info"]["steps"]
            st = srv.stats()
            assert st["completed"] == len(tickets) and st["failed"] == 0
            if rows:
                assert st["packed_requests"] == len(tickets)
                # a chunk serves every waiting member: far fewer chunks than
                # the members' chunks together
                assert 0 < st["packed_chunks"] < steps // params["check_every"]
            else:
                assert st["packed_requests"] == 0 and st["packed_chunks"] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_server_pack_holds_every_product_class(ctx, precision):
    # one pack serves requests of every product class at once -- 200-qubit
    # Ising (group scan, four key words), 4x4 XXZ (group scan, one word) and
    # an 8-orbital product subspace (factored product) -- with members
    # joining and leaving at chunk boundaries; each result equals the
    # request alone (the single product takes the same path class)
    import paper_2603_18731_gb300 as q
    cases = []
    op = wl.ising_heavy_hex(200, seed=4)
    cases.append(("ising200", op, wl.flip_subspace(200, 3000, max_flips=8, seed=2)))
    op = wl.xxz_square(4, 4)
    cases.append(("xxz", op, wl.xxz_walk_subspace(4, 4, count=1500, max_len=8, seed=3)))
    h1, eri = wl.chem_integrals(8, seed=6)
    op = wl.molecular_qubit_operator(h1, eri)
    a = wl.excitation_strings(8, 3, 40, 3, 11)
    b = wl.excitation_strings(8, 3, 30, 3, 12)
    cases.append(("chem8", op, wl.product_subspace(a, b, 8)))
    handles = [(name, ctx.load_operator(op), ctx.build_subspace(op.n_qubits, w)) for name, op, w in cases]
    assert ctx.product_path(handles[2][1], handles[2][2], precision) == 7
    params = dict(precision=precision, max_steps=200, tol=1e-9, check_every=10)
    alone = {name: ctx.lanczos_ground_state(h, s, **params)[0] for name, h, s in handles}
    with q.Server(ctx, budget_bytes=1 << 30, max_active=12) as srv:
        srv.set_pack_rows(1 << 20)
        tickets = []
        for rep in range(3):
            for name, h, s in handles:
                tickets.append((name, srv.submit(h, s, **params)))
            time.sleep(0.002)  # later members join a pack already running
        for name, t in tickets:
            r = srv.wait(t, timeout_s=120)
            assert r["status"] == "OK", (name, r)
            assert abs(r["energy"] - alone[name]) <= 1e-12 * abs(alone[name]), (name, r["energy"], alone[name])
        st = srv.stats()
        assert st["packed_requests"] == len(tickets) and st["failed"] == 0
        assert st["packed_chunks"] > 0
