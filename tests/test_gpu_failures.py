"""Failure handling of the solvers and the served loop, made on the host.

None of these faults, traps or stalls a GPU: allocation failures are
injected in the library's allocator (no CUDA call is made for them), time
limits and waits run out on the host, and the non-convergence and
non-Hermitian cases are ordinary inputs.  After each failure the context
(or the server) must still serve the next request correctly.
"""
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


@pytest.fixture(scope="module")
def xxz(ctx):
    op = wl.xxz_square(4, 4)
    words = wl.xxz_walk_subspace(4, 4, count=2000, max_len=8, seed=5)
    e_ref = oracle.ground_energy(op, oracle.sort_unique(words))
    return ctx.load_operator(op), ctx.build_subspace(16, words), e_ref


@pytest.fixture(autouse=True)
def no_injection():
    import paper_2603_18731_gb300 as q
    yield
    q.lib().qsd_inject_alloc_failures(0)


def test_lanczos_not_converged_returns_best_estimate(ctx, xxz):
    h, sub, e_ref = xxz
    e, info = ctx.lanczos_ground_state(h, sub, check=False, max_steps=4, check_every=2, tol=1e-12)
    assert info["status"] == 7  # QSD_ERR_NOT_CONVERGED
    assert np.isfinite(e) and e >= e_ref - 1e-12 * abs(e_ref)  # a Ritz value lies above E0
    assert info["steps"] == 4 and info["residual"] > 1e-12
    # the context still solves to convergence afterwards
    e2, info2 = ctx.lanczos_ground_state(h, sub, max_steps=300, tol=1e-10)
    assert info2["status"] == 0 and abs(e2 - e_ref) <= 1e-10 * abs(e_ref)


def test_lanczos_time_limit(ctx, xxz):
    h, sub, e_ref = xxz
    e, info = ctx.lanczos_ground_state(h, sub, check=False, max_steps=300, check_every=2, tol=1e-14,
                                       time_limit_s=1e-9)
    assert info["status"] == 8  # QSD_ERR_TIMEOUT
    assert np.isfinite(e) and e >= e_ref - 1e-12 * abs(e_ref)


def test_lanczos_rejects_non_hermitian(ctx):
    import paper_2603_18731_gb300 as q
    op = wl.QubitOperator.from_terms(3, [(1.0, [(0, "+")]), (0.5, [(1, "Z")])])
    h = ctx.load_operator(op)
    assert h.info()["is_hermitian"] == 0
    sub = ctx.build_subspace(3, wl.full_space(3))
    with pytest.raises(q.QsdError) as e:
        ctx.lanczos_ground_state(h, sub)
    assert e.value.status == "NOT_HERMITIAN"


def test_injected_allocation_failure_then_recovery(ctx, xxz):
    import paper_2603_18731_gb300 as q
    h, sub, e_ref = xxz
    assert q.lib().qsd_inject_alloc_failures(-1) == 1  # INVALID_ARG
    q.lib().qsd_inject_alloc_failures(1)
    with pytest.raises(q.QsdError) as e:
        ctx.lanczos_ground_state(h, sub, max_steps=300, tol=1e-10)
    assert e.value.status == "OOM"
    assert b"injected" in q.lib().qsd_last_error(ctx.handle)
    # the failure is used up: the same call succeeds on the same context
    e2, info = ctx.lanczos_ground_state(h, sub, max_steps=300, tol=1e-10)
    assert info["status"] == 0 and abs(e2 - e_ref) <= 1e-10 * abs(e_ref)
    # a subspace build that meets a failure leaves nothing behind
    q.lib().qsd_inject_alloc_failures(1)
    with pytest.raises(q.QsdError) as e:
        ctx.build_subspace(16, wl.xxz_walk_subspace(4, 4, count=500, max_len=6, seed=9))
    assert e.value.status == "OOM"
    assert ctx.build_subspace(16, wl.xxz_walk_subspace(4, 4, count=500, max_len=6, seed=9)).dim > 0


def test_server_admission_after_injected_failure(ctx, xxz):
    import paper_2603_18731_gb300 as q
    h, sub, e_ref = xxz
    with q.Server(ctx, budget_bytes=1 << 28, max_active=2) as srv:
        q.lib().qsd_inject_alloc_failures(1)
        bad = srv.submit(h, sub, max_steps=300, tol=1e-10)
        r = srv.wait(bad, timeout_s=60)
        assert r["status"] == "OOM"
        # its slot and budget are back: later requests are admitted and succeed
        good = [srv.submit(h, sub, max_steps=300, tol=1e-10) for _ in range(3)]
        for t in good:
            r = srv.wait(t, timeout_s=60)
            assert r["status"] == "OK" and abs(r["energy"] - e_ref) <= 1e-10 * abs(e_ref)
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 3
        # retirement follows the results: the budget returns to zero shortly
        t0 = time.time()
        while srv.stats()["bytes_in_use"] and time.time() - t0 < 10:
            time.sleep(0.01)
        assert srv.stats()["bytes_in_use"] == 0


def test_server_wait_timeout_and_request_time_limit(ctx):
    import paper_2603_18731_gb300 as q
    op = wl.ising_heavy_hex(200, seed=4)
    words = wl.flip_subspace(200, 200_000, max_flips=20, seed=8)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(200, words)
    with q.Server(ctx, budget_bytes=1 << 32, max_active=2) as srv:
        t = srv.submit(h, sub, max_steps=300, tol=1e-13, check_every=5)
        r = srv.wait(t, timeout_s=1e-6)
        assert r["status"] == "TIMEOUT"  # the wait ran out, not the request
        r = srv.wait(t, timeout_s=120)
        assert r["status"] in ("OK", "NOT_CONVERGED")
        # a request's own wall-clock limit ends it with its estimate
        t2 = srv.submit(h, sub, max_steps=300, tol=1e-14, check_every=2, time_limit_s=1e-9)
        r2 = srv.wait(t2, timeout_s=120)
        assert r2["status"] == "TIMEOUT" and np.isfinite(r2["energy"])


def test_server_request_above_budget_runs_alone(ctx, xxz):
    import paper_2603_18731_gb300 as q
    h, sub, e_ref = xxz
    # each request's footprint (about 300 Krylov vectors of 2000 rows) is
    # above the whole budget: they are admitted one at a time
    with q.Server(ctx, budget_bytes=1 << 20, max_active=4) as srv:
        tickets = [srv.submit(h, sub, max_steps=300, tol=1e-10) for _ in range(3)]
        res = [srv.wait(t, timeout_s=60) for t in tickets]
        for r in res:
            assert r["status"] == "OK" and abs(r["energy"] - e_ref) <= 1e-10 * abs(e_ref)
        spans = sorted((r["t_admit"], r["t_done"]) for r in res)
        for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
            assert a1 >= d0  # no two ran at once
        st = srv.stats()
        assert st["peak_bytes"] > st["budget_bytes"]
