"""The allocation-free Rayleigh quotient, for callers that cannot call
cudaMalloc: host programs whose own memory pool owns the whole device, and
serving loops that reserve memory up front because cudaMalloc and cudaFree can
synchronise the device mid-flight.

Called through the C ABI and checked against qsd_rayleigh_quotient, which
allocates its scratch, on two calls in a row (the shared fixed scratch keeps
the previous call's contents, which must not leak into the next result); the
device's free memory is unchanged across a warm call; and its size limit.
Kept in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _abi_rq(ctx, name, h, sub, u):
    import paper_2603_18731_gb300 as q
    out = np.zeros(3)
    rc = getattr(q.lib(), name)(ctx.handle, h.handle, sub.handle, ctypes.c_void_p(u.data_ptr()),
                                out.ctypes.data_as(ctypes.c_void_p))
    return rc, out


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    import paper_2603_18731_gb300 as q
    with q.create(0) as ctx:
        op = wl.xxz_square(4, 4)
        words = wl.xxz_walk_subspace(4, 4, count=3000, max_len=8, seed=6)
        h = ctx.load_operator(op)
        sub = ctx.build_subspace(16, words)
        rng = np.random.default_rng(11)
        for call in range(2):
            with torch.cuda.stream(ctx.stream):
                u = torch.as_tensor(rng.normal(size=sub.dim), device=ctx.device)
            rc_a, ref = _abi_rq(ctx, "qsd_rayleigh_quotient", h, sub, u)
            rc_b, got = _abi_rq(ctx, "qsd_rayleigh_quotient_noalloc", h, sub, u)
            assert rc_a == 0 and rc_b == 0, (call, rc_a, rc_b)
            assert abs(got[0] - ref[0]) <= TOL * abs(ref[0]), (call, got, ref)
            assert abs(got[1] - ref[1]) <= 1e-10 * abs(ref[1]), (call, got, ref)
            assert abs(got[2] - ref[2]) <= TOL * abs(ref[2]), (call, got, ref)


def test_noalloc_leaves_device_free_memory_unchanged():
    import torch
    import paper_2603_18731_gb300 as q
    with q.create(0) as ctx:
        op = wl.ising_heavy_hex(60, seed=9)
        words = wl.flip_subspace(60, 20_000, max_flips=8, seed=9)
        h = ctx.load_operator(op)
        sub = ctx.build_subspace(60, words)
        with torch.cuda.stream(ctx.stream):
            u = torch.as_tensor(np.random.default_rng(3).normal(size=sub.dim), device=ctx.device)
        # the first call loads the kernels and resolves the scratch address
        rc, first = _abi_rq(ctx, "qsd_rayleigh_quotient_noalloc", h, sub, u)
        assert rc == 0
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc, again = _abi_rq(ctx, "qsd_rayleigh_quotient_noalloc", h, sub, u)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert rc == 0
        assert free1 == free0, (free0, free1)
        assert np.array_equal(first, again)


def test_noalloc_rejects_subspace_above_limit():
    import torch
    import paper_2603_18731_gb300 as q
    with q.create(0) as ctx:
        op = wl.tfim_chain(21, g=1.0)
        h = ctx.load_operator(op)
        sub = ctx.build_subspace(21, wl.full_space(21))
        assert sub.dim == 1 << 21
        with torch.cuda.stream(ctx.stream):
            u = torch.ones(sub.dim, dtype=torch.float64, device=ctx.device)
        rc, _ = _abi_rq(ctx, "qsd_rayleigh_quotient_noalloc", h, sub, u)
        assert q.STATUS[rc] == "CAPACITY"
        assert b"at most" in q.lib().qsd_last_error(ctx.handle)


def test_noalloc_factored_pair_builds_no_tables():
    # a product subspace with linear ranges: the allocating products build
    # per-pair half-sum tables on first use; the allocation-free entry point
    # must not, even on a pair it has never seen (its kernels are loaded by a
    # first call on another subspace of the same operator), and gives the
    # same quotient
    import torch
    import paper_2603_18731_gb300 as q
    with q.create(0) as ctx:
        h1, eri = wl.chem_integrals(8, seed=4)
        op = wl.molecular_qubit_operator(h1, eri)
        h = ctx.load_operator(op)
        assert h.info()["n_linear_ranges"] > 0
        strings = [v for v in range(1 << 8) if bin(v).count("1") == 3]
        warm = ctx.build_subspace(16, wl.product_subspace(strings[:30], strings[:20], 8))
        sub = ctx.build_subspace(16, wl.product_subspace(strings, strings[:40], 8))
        assert sub.factored()["is_product"] and ctx.product_path(h, sub) == 7
        rng = np.random.default_rng(5)
        with torch.cuda.stream(ctx.stream):
            uw = torch.as_tensor(rng.normal(size=warm.dim), device=ctx.device)
            u = torch.as_tensor(rng.normal(size=sub.dim), device=ctx.device)
        rc, _ = _abi_rq(ctx, "qsd_rayleigh_quotient_noalloc", h, warm, uw)
        assert rc == 0
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc, got = _abi_rq(ctx, "qsd_rayleigh_quotient_noalloc", h, sub, u)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert rc == 0
        assert free1 == free0, (free0, free1)
        rc, ref = _abi_rq(ctx, "qsd_rayleigh_quotient", h, sub, u)  # builds the tables
        assert rc == 0
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0]) and abs(got[2] - ref[2]) <= TOL * abs(ref[2])
