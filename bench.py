"""Benchmark of the subspace Hamiltonian-vector product on one GB300 (or N
replicas under torchrun).

Workload (default): the 2D XXZ model on the 6x6 periodic square lattice
(36 qubits), H = sum_<ij> 0.5 (s+_i s-_j + s-_i s+_j) + Z_i Z_j, over 300,000
distinct weight-18 bit-strings from seeded bond-swap walks (length 1-12) from
the Neel state.  One step = one FP64 product y = H_S x over the whole
subspace (k = 1).  Throughput is Gelem/s = D * (groups + 1) * k / t (the
paper's count of matrix-element evaluations: subspace dimension times the
number of groups, diagonal group included).

Extra objects on the same JSON line: the FP32-mixed and block (k = 16)
variants timed the same way, a full ground-state solve, the roofline of the
product kernel, the CPU oracle baseline, clocks sampled during the timed
region, and the end-to-end number through the host-buffer ABI call.

  python bench.py [--steps K] [--warmup W] [--workload xxz|tfim|ising]
  python bench.py --impl reference      # the CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

if "OMP_NUM_THREADS" not in os.environ:
    os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "apply_H Gelem/s FP64 vs FP32-mixed block; served eigensolves/s, p50/p99 latency"
L2_FLUSH_BYTES = 512 << 20
PATH_NAMES = {0: "group scan, lane per row", 1: "group scan, 8 lanes per row", 2: "excitation index",
              3: "half evaluation, lane per row", 4: "half evaluation, 8 lanes per row",
              5: "group scan, lane per row, rows in hash order",
              6: "half evaluation, lane per row, rows in hash order",
              7: "sector-factored enumeration, warp per row"}


# ------------------------------------------------------------------ workloads
def make_workload(name: str):
    if name == "xxz":
        op = wl.xxz_square(6, 6, 0.5, 1.0)
        words = wl.xxz_walk_subspace(6, 6, count=300_000, max_len=12, seed=2)
        desc = ("2D XXZ 6x6 periodic (36 qubits), 300k distinct weight-18 strings from bond-swap walks "
                "(len 1-12) from Neel, seed 2")
    elif name == "tfim":
        op = wl.tfim_chain(12, g=1.0)
        words = wl.full_space(12)
        desc = "1D TFIM 12 qubits periodic, full 4096-string space"
    elif name == "ising":
        op = wl.ising_heavy_hex(200, seed=4)
        words = wl.flip_subspace(200, 1_000_000, max_flips=20, seed=4)
        desc = "Ising 200 qubits heavy-hex-like graph, 1M strings = seeded reference with 1-20 bits flipped"
    elif name == "chem":
        h1, eri = wl.chem_integrals(32, seed=3)
        op = wl.molecular_qubit_operator(h1, eri)
        alpha = wl.excitation_strings(32, 8, 1500, 4, seed=3)
        beta = wl.excitation_strings(32, 8, 1500, 4, seed=1003)
        words = wl.product_subspace(alpha, beta, 32)
        desc = ("fermionic 32 spatial orbitals (64 qubits, extended JW), h ~ N(0,0.1), (pq|rs) ~ N(0,0.05) "
                "exp(-|p-q|-|r-s|), S = 1500 alpha x 1500 beta weight-8 strings (HF + 1-4 excitations), seed 3")
    else:
        raise SystemExit(f"unknown workload {name}")
    return op, words, desc


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def read_profile_traffic(kernel_tag: str):
    """Per-launch DRAM bytes of the product kernel from the committed ncu
    summary (profiles/<tag>.md, line 'traffic_bytes_per_launch: N'), or None."""
    p = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith("traffic_bytes_per_launch:"):
            v = line.split(":", 1)[1].strip()
            return None if v in ("", "null", "None") else float(v)
    return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over the ranks of the default process group (x itself
    when there is none)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Units processed by all ranks (each does the same work) per second of
    the slowest rank."""
    return world * units_per_rank / seconds


def run_gpu(args):
    import torch
    import paper_2603_18731_gb300 as q

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    op, words, desc = make_workload(args.workload)
    ctx = q.create(local)
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    info = h.info()
    D, G, W = sub.dim, info["n_groups"], sub.W
    dev = ctx.device
    s = ctx.stream
    rng = np.random.default_rng(0)
    with torch.cuda.stream(s):
        x64 = torch.as_tensor(rng.normal(size=D), device=dev)
        x32 = x64.float()
        xb64 = torch.as_tensor(rng.normal(size=(D, 16)), device=dev)
        xb32 = xb64.float()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # lookups / hits per product (integer target table, not timed); sampled
    # rows, scaled to D, when the full table would exceed 2^31 entries
    lookups = hits = 0
    chunk = max(1, (1 << 27) // max(G, 1))
    sampled = D * G > (1 << 31)
    starts = (np.linspace(0, D - 1, 64).astype(int).tolist() if sampled else list(range(0, D, chunk)))
    nrow = 0
    for r0 in starts:
        n = min(chunk if not sampled else max(1, (1 << 24) // max(G, 1)), D - r0)
        tt = ctx.target_table(h, sub, r0, n)
        ctx.synchronize()
        lookups += int((tt != -2).sum().item())
        hits += int((tt >= 0).sum().item())
        nrow += n
        del tt
    if sampled:
        lookups = int(lookups * D / nrow)
        hits = int(hits * D / nrow)
    ctx.synchronize()

    def time_variant(x, precision, steps, warmup):
        y = ctx.empty(tuple(x.shape), x.dtype)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for _ in range(warmup):
            ctx.apply_H(h, sub, x, y, precision)
        ctx.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            with torch.cuda.stream(s):
                flush.zero_()
            ev[i][0].record(s)
            ctx.apply_H(h, sub, x, y, precision)
            ev[i][1].record(s)
        ctx.synchronize()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in ev]
        return float(np.mean(ms)), ms, wall

    elems = D * (G + 1)
    # headline: FP64, k = 1 -- except the fermionic workload, whose
    # configuration is the k = 16 block with FP32 storage and FP64 accumulation
    head_x, head_prec, k1 = (xb32, q.QSD_FP32_MIXED, 16) if args.workload == "chem" else (x64, q.QSD_FP64, 1)
    with ClockSampler(local) as clk:
        ms64, all64, wall64 = time_variant(head_x, head_prec, args.steps, args.warmup)
    # replicas: the job takes as long as its slowest rank
    t_max = max_over_ranks(ms64, dist, dev)
    value = whole_job_rate(elems * k1, t_max * 1e-3, world) / 1e9
    variants = {}
    vsteps = max(3, min(args.steps, 20))
    vlist = [("fp32_mixed_k1", x32, q.QSD_FP32_MIXED, 1), ("fp32_dot2_k1", x32, q.QSD_FP32_DOT2, 1),
             ("fp64_k16", xb64, q.QSD_FP64, 16), ("fp32_mixed_k16", xb32, q.QSD_FP32_MIXED, 16),
             ("fp32_dot2_k16", xb32, q.QSD_FP32_DOT2, 16)]
    if args.workload == "chem":
        vlist = [("fp64_k1", x64, q.QSD_FP64, 1), ("fp32_mixed_k16", xb32, q.QSD_FP32_MIXED, 16),
                 ("fp32_dot2_k16", xb32, q.QSD_FP32_DOT2, 16)]
        vsteps = 3
    for name, x, prec, k in vlist:
        m, _, _ = time_variant(x, prec, vsteps, 3)
        variants[name] = {"ms": m, "gelem_s": elems * k / (m * 1e-3) / 1e9}
    if info["is_hermitian"] and info["is_real"] and W <= 4:
        # half evaluation: lower-triangle groups by MSOB, mirrored by FP64
        # atomic adds (summation order varies between runs)
        ctx.set_tuning(1, 3)
        for name, x, k in (("fp64_k1_half", x64, 1), ("fp64_k16_half", xb64, 16)):
            for lanes, order, tag in ((1, 1, "lanes1"), (8, 1, "lanes8"), (1, 2, "hash_order")):
                ctx.set_tuning(2, lanes)
                ctx.set_tuning(5, order)
                m, _, _ = time_variant(x, q.QSD_FP64, vsteps, 3)
                variants[f"{name}_{tag}"] = {"ms": m, "gelem_s": elems * k / (m * 1e-3) / 1e9}
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.set_tuning(5, 0)
    if args.workload != "chem" and W <= 4:
        # every group-scan launch shape, forced (the tuner picks among these)
        ctx.set_tuning(1, 1)
        for name, x, prec, k in (("fp64_k1", x64, q.QSD_FP64, 1), ("fp32_mixed_k16", xb32, q.QSD_FP32_MIXED, 16)):
            for lanes, order, tag in ((1, 1, "lanes1"), (8, 1, "lanes8"), (1, 2, "hash_order")):
                ctx.set_tuning(2, lanes)
                ctx.set_tuning(5, order)
                m, _, _ = time_variant(x, prec, vsteps, 3)
                variants[f"{name}_scan_{tag}"] = {"ms": m, "gelem_s": elems * k / (m * 1e-3) / 1e9}
        ctx.set_tuning(1, 0)
        ctx.set_tuning(2, 0)
        ctx.set_tuning(5, 0)
    fp64_1 = (variants["fp64_k1"]["gelem_s"] if args.workload == "chem" else elems / (ms64 * 1e-3) / 1e9)
    variants["mixed_block_over_fp64"] = variants["fp32_mixed_k16"]["gelem_s"] / fp64_1
    variants["dot2_block_over_fp64"] = variants["fp32_dot2_k16"]["gelem_s"] / fp64_1

    # roofline of the headline product kernel: algorithmic bytes
    s_x = 8 * k1 if head_prec == q.QSD_FP64 else 4 * k1
    b_alg = D * (W * 8 + 8 + s_x + s_x) + lookups * 8 + hits * (W * 8 + s_x)
    b_alg += info["n_terms"] * (3 * W * 8 + 8 + 1) + G * (W * 8 + 8 + 4 + 1 + 8 + 68)
    peak, peak_kind = load_peaks()
    achieved = b_alg / (ms64 * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} hbm_gbs (burst, kernel timed alone)",
            "traffic": read_profile_traffic(f"apply_H_{args.workload}"),
            "algorithmic_bytes_per_launch": b_alg, "lookups_per_launch": lookups, "hits_per_launch": hits}

    # end to end through the host-buffer ABI call (pinned host memory)
    hdt = torch.float64 if head_prec == q.QSD_FP64 else torch.float32
    xh = torch.empty(tuple(head_x.shape), dtype=hdt, pin_memory=True).numpy()
    xh[:] = head_x.cpu().numpy()
    yh = torch.empty(tuple(head_x.shape), dtype=hdt, pin_memory=True).numpy()
    for _ in range(args.warmup):
        ctx.apply_H_host(h, sub, xh, head_prec, out=yh)
    et = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ctx.apply_H_host(h, sub, xh, head_prec, out=yh)
        et.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(et)), dist, dev)
    e2e = {"value": whole_job_rate(elems * k1, e2e_s, world) / 1e9, "unit": "Gelem/s",
           "h2d_bytes_per_step": int(xh.nbytes),
           "d2h_bytes_per_step": int(yh.nbytes), "ms_per_step": e2e_s * 1e3}

    # one full ground-state solve per precision (not part of the timed steps)
    solve = {}
    if not args.no_solve:
        for name, prec in (("fp64", q.QSD_FP64), ("fp32_mixed", q.QSD_FP32_MIXED), ("fp32_dot2", q.QSD_FP32_DOT2)):
            ctx.synchronize()
            t0 = time.perf_counter()
            e, inf = ctx.lanczos_ground_state(h, sub, check=False, precision=prec, max_steps=args.solve_steps,
                                              tol=1e-9)
            ctx.synchronize()
            solve[name] = {"seconds": time.perf_counter() - t0, "energy": e, "steps": inf["steps"],
                           "applies": inf["applies"], "residual": inf["residual"], "status": inf["status"]}

    # explicit CSR build: lower triangle by MSOB and mirror, against every
    # group of every row (two passes each, device sort of the entries)
    csr = None
    if not args.no_csr and args.workload != "chem":
        csr = {}
        for name, full in (("msob_lower", False), ("full", True)):
            ts, tc = [], []
            for rep in range(4):
                ctx.synchronize()
                t0 = time.perf_counter()
                nnz = ctx.csr_size(h, sub, full=full)  # pass 1 (kept for the fill)
                t1 = time.perf_counter()
                ip, ind, dat = ctx.to_csr(h, sub, full=full)
                ctx.synchronize()
                if rep:
                    ts.append(time.perf_counter() - t0)
                    tc.append(t1 - t0)
                del ip, ind, dat
            csr[name] = {"ms": 1e3 * float(np.mean(ts)), "count_pass_ms": 1e3 * float(np.mean(tc)), "nnz": nnz}
        csr["msob_speedup"] = csr["full"]["ms"] / csr["msob_lower"]["ms"]

    # block LOBPCG (shifted Jacobi preconditioner, the paper's spiked start),
    # 4 lowest eigenpairs
    lob = None
    if not args.no_solve and args.workload != "chem":
        lob = {}
        for pre in (1, 0):
            ctx.synchronize()
            t0 = time.perf_counter()
            ev, inf = ctx.lobpcg(h, sub, k=4, tol=1e-8, precondition=pre, max_iters=600, check=False)
            ctx.synchronize()
            lob["jacobi" if pre else "none"] = {"seconds": time.perf_counter() - t0, "evals": ev.tolist(),
                                                "iters": inf["iters"], "status": inf["status"],
                                                "max_residual": inf["max_residual"]}

    # RAMPS refinement from one reference bit-string (the lowest-diagonal
    # row of the workload's subspace), E = its diagonal, unrestricted
    ramps_out = None
    if not args.no_ramps and W <= 4 and args.workload != "chem":
        ramps_out = run_ramps(ctx, h, sub, op, args.ramps_tau)

    # packed launches: many small products (64 walk subspaces of the
    # workload's family, D log-uniform in [500, 5000]) as one launch against
    # one launch per pair
    packed = None
    if not args.no_packed and W <= 4 and args.workload != "chem":
        packed = run_packed(ctx, q, op, args.workload)

    serve = None
    if not args.no_serve:
        serve = run_serve(args, q, local)
        if args.serve_compare:
            other = 0 if args.serve_pack_rows else 32768
            serve["compare_pack_rows_%d" % other] = run_serve(args, q, local, pack_rows=other)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(op, words, G, target_seconds=args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head_prec == q.QSD_FP64 else "f32+f64acc", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "dim": D, "groups": G, "qubits": op.n_qubits,
                       "k": k1, "precision": "fp64" if head_prec == q.QSD_FP64 else "fp32 storage, fp64 accumulation",
                       "product_path": PATH_NAMES[ctx.product_path(h, sub, head_prec, k1)],
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": args.steps, "roofline": roof, "cpu_baseline": cpu,
            "clocks": clk.summary(), "variants": variants, "solve": solve, "lobpcg_k4": lob, "csr_build": csr, "ramps": ramps_out, "packed": packed, "serve": serve,
            "step_ms_min_max": [float(np.min(all64)), float(np.max(all64))],
        }
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_ramps(ctx, h, sub, op, tau, max_levels=8, reps=3):
    import torch
    d = ctx.diagonal(h, sub)
    r0 = int(torch.argmin(d).item())
    E = float(d[r0].item())
    keys = ctx.subspace_keys(sub)[r0:r0 + 1]
    start = ctx.build_subspace(op.n_qubits, keys)
    ts, out, info = [], None, None
    for rep in range(reps + 1):
        ctx.synchronize()
        t0 = time.perf_counter()
        out, info = ctx.ramps(h, start, E, tau, max_levels=max_levels, max_rows=4_000_000)
        ctx.synchronize()
        if rep:
            ts.append(time.perf_counter() - t0)
        if rep < reps:
            out.free()
    G = h.info()["n_groups"]
    # rows expanded: the start row and every level's rows, except the last
    # level's when the level or row limit ended the recursion
    lr = info["level_rows"]
    pairs = 1 + sum(lr) - (lr[-1] if lr and (info["stopped_by_limit"] or info["truncated"]) else 0)
    ms = 1e3 * float(np.mean(ts))
    res = {"tau": tau, "E": E, "ms": ms, "rows_out": info["rows_out"], "levels": info["levels"],
           "level_rows": info["level_rows"], "candidates": info["candidates"],
           "stopped_by_limit": info["stopped_by_limit"], "truncated": info["truncated"],
           "row_group_pairs_per_s": pairs * G / (ms * 1e-3)}
    out.free()
    start.free()
    return res


def run_packed(ctx, q, op, workload, n_pairs=64, reps=20):
    import torch
    rng = np.random.default_rng(11)
    h = ctx.load_operator(op)
    subs, xs = [], []
    for i in range(n_pairs):
        d = int(np.exp(rng.uniform(np.log(500), np.log(5000))))
        if workload == "xxz":
            words = wl.xxz_walk_words(6, 6, d, 12, 100 + i)
        elif workload == "tfim":
            words = wl.random_subspace(op.n_qubits, d, seed=100 + i)
        else:
            words = wl.flip_words(op.n_qubits, d, 20, 100 + i)
        s_ = ctx.build_subspace(op.n_qubits, words)
        subs.append(s_)
        with torch.cuda.stream(ctx.stream):
            xs.append(torch.as_tensor(rng.normal(size=s_.dim), device=ctx.device))
    ops = [h] * n_pairs
    ys = [ctx.empty((s_.dim,), torch.float64) for s_ in subs]
    G = h.info()["n_groups"]
    elems = sum(s_.dim for s_ in subs) * (G + 1)
    ctx.set_tuning(1, 1)
    ctx.set_tuning(2, 1)

    def timed(fn):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(ctx.stream)
            fn()
            b.record(ctx.stream)
        ctx.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    t_single = timed(lambda: [ctx.apply_H(h, s_, x, y) for s_, x, y in zip(subs, xs, ys)])
    t_packed = timed(lambda: ctx.apply_H_batch(ops, subs, xs, ys))
    ctx.set_tuning(1, 0)
    ctx.set_tuning(2, 0)
    return {"pairs": n_pairs, "rows": int(sum(s_.dim for s_ in subs)), "one_launch_per_pair_ms": t_single,
            "packed_ms": t_packed, "packed_gelem_s": elems / (t_packed * 1e-3) / 1e9,
            "one_launch_per_pair_gelem_s": elems / (t_single * 1e-3) / 1e9, "speedup": t_single / t_packed}


# ------------------------------------------------------------------ serving
def serve_pool(n_pool: int, seed: int, dmin: float, dmax: float):
    """Workloads for the served stream: the three families, each with fresh
    seeds and a log-uniform target dimension.  Host generation only; each
    request does its own device build (sort, dedup, hash, grouping)."""
    rng = np.random.default_rng(seed)
    pool = []
    ferm_ops = {}
    for i in range(n_pool):
        fam = ("ising", "xxz", "fermion")[i % 3]
        s_ = int(rng.integers(1, 1 << 30))
        target = int(np.exp(rng.uniform(np.log(dmin), np.log(dmax))))
        if fam == "ising":
            op = wl.ising_heavy_hex(200, seed=s_ % 1000)
            words = wl.flip_words(200, target, 20, s_)
        elif fam == "xxz":
            op = wl.xxz_square(6, 6)
            words = wl.xxz_walk_words(6, 6, target, 12, s_)
        else:
            n_orb, ne = 8, 4
            key = s_ % 4
            if key not in ferm_ops:
                h1, eri = wl.chem_integrals(n_orb, seed=1000 + key)
                ferm_ops[key] = wl.molecular_qubit_operator(h1, eri)
            op = ferm_ops[key]
            side = int(min(70, max(2, round(np.sqrt(target)))))
            alpha = wl.excitation_strings(n_orb, ne, side, 4, s_)
            beta = wl.excitation_strings(n_orb, ne, side, 4, s_ + 1)
            words = wl.product_subspace(alpha, beta, n_orb)
        pool.append((fam, op, words))
    return pool


def run_serve(args, q, local, pack_rows=None):
    """512 Poisson arrivals at 0.8x the measured closed-loop capacity; latency
    from arrival to energy ready, including the request's device build."""
    import torch
    pack_rows = args.serve_pack_rows if pack_rows is None else pack_rows
    rng = np.random.default_rng(args.serve_seed)
    pool = serve_pool(args.serve_pool, args.serve_seed, 1e3, 2e6)
    client = q.create(local)
    srvctx = q.create(local)
    budget = int(args.serve_budget_gb * (1 << 30))
    params = dict(precision=q.QSD_FP32_DOT2, max_steps=300, tol=1e-7, check_every=10)
    handles = []

    def build(i):
        fam, op, words = pool[i]
        h = client.load_operator(op)
        sub = client.build_subspace(op.n_qubits, words)
        handles.append((h, sub))
        return h, sub

    def run(order, arrivals, srv, host_t0):
        tickets = [None] * len(order)
        t_arr = [0.0] * len(order)
        start = time.perf_counter()

        def feeder():
            for k, i in enumerate(order):
                delay = start + arrivals[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                t_arr[k] = time.perf_counter()
                h, sub = build(i)
                tickets[k] = srv.submit(h, sub, **params)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        res = []
        for k, t in enumerate(tickets):
            r = srv.wait(t)
            r["latency_s"] = host_t0 + r["t_done"] - t_arr[k]
            r["build_s"] = host_t0 + r["t_submit"] - t_arr[k]
            r["queue_s"] = r["t_admit"] - r["t_submit"]
            r["run_s"] = r["t_done"] - r["t_admit"]
            r["family"] = pool[order[k]][0]
            res.append(r)
        wall = time.perf_counter() - start
        return res, wall

    with q.Server(srvctx, budget_bytes=budget, max_active=args.serve_slots) as srv:
        srv.set_pack_rows(pack_rows)
        host_t0 = time.perf_counter()
        # closed-loop capacity: every pool item submitted at once
        burst, t_burst = run(list(range(len(pool))), [0.0] * len(pool), srv, host_t0)
        capacity = len(pool) / t_burst
        lam = 0.8 * capacity
        n = args.serve_requests
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n)).tolist()
        order = rng.integers(0, len(pool), size=n).tolist()
        res, wall = run(order, arrivals, srv, host_t0)
        st = srv.stats()
    lat = np.array([r["latency_s"] for r in res]) * 1e3
    ok = [r for r in res if r["status"] == "OK"]
    phases = {f"{ph}_p50_ms": float(np.percentile([r[f"{ph}_s"] for r in res], 50)) * 1e3
              for ph in ("build", "queue", "run")}
    fams = {}
    for r in res:
        fams.setdefault(r["family"], []).append(r["latency_s"] * 1e3)
    dims = [pool[i][2].shape[0] for i in order]
    out = {"requests": n, "ok": len(ok), "rate_hz": lam, "closed_loop_capacity_solves_s": capacity,
           "solves_per_s": len(ok) / wall, "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
           "max_active": args.serve_slots, "budget_bytes": budget, "peak_bytes": st["peak_bytes"],
           "per_family_p50_ms": {k: float(np.percentile(v, 50)) for k, v in fams.items()},
           "phases": phases, "pack_rows": pack_rows,
           "packed_requests": st["packed_requests"], "packed_chunks": st["packed_chunks"],
           "candidate_dims_min_max": [int(min(dims)), int(max(dims))],
           "precision": "fp32_dot2 + fp64 refinement", "tol": params["tol"],
           "note": "latency = arrival to energy ready, including the request's device subspace build "
                   "and operator grouping; host synthetic generation excluded (pool of %d workloads)" % len(pool)}
    client.close()
    srvctx.close()
    return out


# ------------------------------------------------------------------ CPU arm
def cpu_baseline(op, words, G, target_seconds=12.0, sample_rows=None):
    """The plain oracle product on a bounded sample of rows, timed on the host
    cores; returns Gelem/s on the same count (rows * (groups + 1))."""
    import oracle
    keys = oracle.sort_unique(words)
    D = keys.shape[0]
    x = np.random.default_rng(0).normal(size=D)
    rng = np.random.default_rng(1)
    n = min(D, 512)
    rows = np.sort(rng.choice(D, size=n, replace=False))
    t0 = time.perf_counter()
    oracle.apply_rows(op, keys, x, rows)
    dt = max(time.perf_counter() - t0, 1e-6)
    if sample_rows is None:
        sample_rows = int(min(D, max(n, n * target_seconds / dt)))
    rows = np.sort(rng.choice(D, size=sample_rows, replace=False))
    t0 = time.perf_counter()
    oracle.apply_rows(op, keys, x, rows)
    dt = time.perf_counter() - t0
    return {"value": sample_rows * (G + 1) / dt / 1e9, "unit": "Gelem/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "seconds": dt,
            "sample": f"{sample_rows} of {D} rows (uniform sample), FP64 product, OpenMP over rows"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    op, words, desc = make_workload(args.workload)
    keys = oracle.sort_unique(words)
    # group count by the oracle's own definition (distinct flip sets)
    G = oracle.groups(op).shape[0]
    D = keys.shape[0]
    x = np.random.default_rng(0).normal(size=D)
    rng = np.random.default_rng(2)
    probe = np.sort(rng.choice(D, size=min(D, 512), replace=False))
    t0 = time.perf_counter()
    oracle.apply_rows(op, keys, x, probe)
    dt = max(time.perf_counter() - t0, 1e-6)
    per_step = args.ref_step_seconds
    n = int(min(D, max(64, len(probe) * per_step / dt)))
    rows = np.sort(rng.choice(D, size=n, replace=False))
    for _ in range(args.warmup):
        oracle.apply_rows(op, keys, x, rows)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.apply_rows(op, keys, x, rows)
        ts.append(time.perf_counter() - t0)
    ms = float(np.mean(ts)) * 1e3
    value = n * (G + 1) / (ms * 1e-3) / 1e9
    cores = int(os.environ["OMP_NUM_THREADS"])
    sample = f"{n} of {D} rows per step (uniform sample), FP64 product, OpenMP over rows"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "dim": D, "groups": G, "k": 1,
                   "precision": "fp64", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="xxz", choices=["xxz", "tfim", "ising", "chem"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--solve-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=2.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-csr", action="store_true", help="skip the CSR build timing")
    ap.add_argument("--no-packed", action="store_true", help="skip the packed-launch timing")
    ap.add_argument("--no-ramps", action="store_true", help="skip the RAMPS timing")
    ap.add_argument("--ramps-tau", type=float, default=1e-7)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-pool", type=int, default=36)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-pack-rows", type=int, default=0,
                    help="requests up to this many rows run in packed chunks (0: never)")
    ap.add_argument("--serve-compare", action="store_true",
                    help="also run the served stream with packing switched the other way")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-seed", type=int, default=5)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
