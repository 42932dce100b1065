"""Benchmark of the subspace Hamiltonian-vector product on one GB300 (or N
replicas under torchrun).

Workload (default, the largest single-GPU configuration): a fermionic
chemistry-like Hamiltonian of 32 spatial orbitals (64 qubits, extended
Jordan-Wigner; seeded integrals h_pq ~ N(0, 0.1), (pq|rs) ~ N(0, 0.05)
exp(-|p-q| - |r-s|) with 8-fold symmetry; 1,542,656 qubit terms in 318,928
groups) over the product of 1500 alpha x 1500 beta weight-8 strings
(2,250,000 rows).  One step = one FP64 product y = H_S X of a block of 16
vectors over the whole subspace.  Throughput is Gelem/s = D * (groups + 1) * k
/ t (the paper's count of matrix-element evaluations: subspace dimension
times the number of groups, diagonal group included, per vector).

Extra objects on the same JSON line: the FP32-mixed (the configuration's
stated form), FP32-DOT2 and single-vector FP64 variants timed the same way,
each with its roofline; a ground-state solve; the end-to-end number through
the host-buffer ABI call; the CPU oracle baseline; clocks sampled during the
timed region; the 200-qubit Ising (1 M rows) and 6x6 XXZ (300,000 rows)
workloads with their own lines (FP64 single-vector headline, block variants,
rooflines, solves, CSR build, LOBPCG, RAMPS, packed launches); the served
stream.

  python bench.py [--steps K] [--warmup W] [--workload chem|xxz|ising|tfim]
  python bench.py --product-only ...    # the headline product steps alone
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
              7: "sector-factored enumeration, warp per row",
              8: "filter/verify scan, lane per row, rows in hash order"}


# ------------------------------------------------------------------ workloads
def make_workload(name: str, chem_strings: int = 1500):
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
        alpha = wl.excitation_strings(32, 8, chem_strings, 4, seed=3)
        beta = wl.excitation_strings(32, 8, chem_strings, 4, seed=1003)
        words = wl.product_subspace(alpha, beta, 32)
        desc = ("fermionic 32 spatial orbitals (64 qubits, extended JW), h ~ N(0,0.1), (pq|rs) ~ N(0,0.05) "
                f"exp(-|p-q|-|r-s|), S = {chem_strings} alpha x {chem_strings} beta weight-8 strings "
                "(HF + 1-4 excitations), seed 3")
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


# product path -> qsd_set_tuning (knob, value) pairs
PATH_KNOBS = {"auto": [], "scan": [(1, 1), (2, 1), (5, 1)], "scan-hash": [(1, 1), (2, 1), (5, 2)],
              "scan8": [(1, 1), (2, 8)], "excitation": [(1, 2)], "factored": [(1, 4)], "filter-verify": [(1, 5)]}
HEAD = {"chem": (0, 16), "xxz": (0, 1), "ising": (0, 1), "tfim": (0, 1)}  # (precision, k)
SPIN_EXTRAS = ("ising", "xxz")


def read_profile(tag: str, path: int):
    """(traffic bytes, warp instructions) per launch from the committed ncu
    summary profiles/<tag>.md ('traffic_bytes_per_launch: N',
    'warp_instructions_per_launch: N', 'product_path: P'), when it profiles
    the product path that was timed; else (None, None)."""
    p = os.path.join(ROOT, "profiles", f"{tag}.md")
    if not os.path.exists(p):
        return None, None
    vals = {}
    for line in open(p):
        for key in ("traffic_bytes_per_launch", "warp_instructions_per_launch", "product_path"):
            if line.startswith(key + ":"):
                v = line.split(":", 1)[1].strip()
                vals[key] = None if v in ("", "null", "None") else float(v)
    if vals.get("product_path") != path:
        return None, None
    return vals.get("traffic_bytes_per_launch"), vals.get("warp_instructions_per_launch")


def algorithmic_bytes(path, D, W, k, s_x, lookups, hits, n_terms, G):
    """Bytes one product must move (per row: key, diagonal, own x and y; per
    lookup: the bucket; per hit: the key check and the gathered x; term and
    group tables once).  The sector-factored path makes no lookups and checks
    no key: per found column it reads its two neighbour entries and its
    rank-index entry (12 bytes) and gathers x."""
    per_row = W * 8 + 8 + 2 * k * s_x
    tables = n_terms * (3 * W * 8 + 8 + 1) + G * (W * 8 + 8 + 4 + 1 + 8 + 68)
    if path == 7:
        return D * per_row + hits * (12 + k * s_x) + tables
    return D * per_row + lookups * 8 + hits * (W * 8 + k * s_x) + tables


class Timer:
    """CUDA-event timing of products on the context's stream, the L2
    flushed (a 512 MiB write) before every timed launch."""

    def __init__(self, ctx, dist=None):
        import torch
        self.torch, self.ctx, self.dist = torch, ctx, dist
        with torch.cuda.stream(ctx.stream):
            self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=ctx.device)

    def time(self, fn, steps, warmup):
        torch, s = self.torch, self.ctx.stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for _ in range(warmup):
            fn()
        self.ctx.synchronize()
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            with torch.cuda.stream(s):
                self.flush.zero_()
            ev[i][0].record(s)
            fn()
            ev[i][1].record(s)
        self.ctx.synchronize()
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return float(np.mean(ms)), ms


def count_lookups(ctx, h, sub, G):
    """Lookups and hits of one single-vector product from the integer target
    table (not timed): every row when the table has at most 2^31 entries,
    else 512 runs of 4 rows at uniformly drawn positions (an unbiased sample:
    rows of one index range share a half-string and their counts are
    correlated), scaled to D."""
    D = sub.dim
    sampled = D * G > (1 << 31)
    if sampled:
        run = 4
        starts = np.sort(np.random.default_rng(7).choice(D - run + 1, size=min(512, D - run + 1), replace=False))
        spans = [(int(r0), run) for r0 in starts]
    else:
        chunk = max(1, (1 << 27) // max(G, 1))
        spans = [(r0, min(chunk, D - r0)) for r0 in range(0, D, chunk)]
    lookups = hits = nrow = 0
    for r0, n in spans:
        tt = ctx.target_table(h, sub, r0, n)
        ctx.synchronize()
        lookups += int((tt != -2).sum().item())
        hits += int((tt >= 0).sum().item())
        nrow += n
        del tt
    if sampled:
        lookups = int(lookups * D / nrow)
        hits = int(hits * D / nrow)
    return lookups, hits, ("sampled %d rows in %d runs at random positions" % (nrow, len(spans))) if sampled \
        else "every row"


FP64_FMA_PER_SM_CYCLE = 2  # GB300: FP64 FMA issue rate per SM per cycle (1/64 of FP32)


def roofline_of(ms, path, tag, D, W, k, prec, lookups, hits, info, peak, peak_kind, sm_mhz, n_sms):
    """Roofline of one product launch.  The sector-factored path with FP64
    accumulation (QSD_FP64, QSD_FP32_MIXED) is bound by the FP64 FMA pipe:
    every found column costs k FP64 FMAs and the GB300 retires 2 per SM per
    cycle, so that bound is reported ('alu', FP64 TFLOP/s at the sampled SM
    clock) with the HBM figures beside it; every other launch by memory
    ('hbm').  A committed ncu summary of the same path adds its measured DRAM
    traffic and the warp-instruction issue roof."""
    s_x = 8 if prec == 0 else 4
    G = info["n_groups"]
    b_alg = algorithmic_bytes(path, D, W, k, s_x, lookups, hits, info["n_terms"], G)
    achieved = b_alg / (ms * 1e-3) / 1e9
    traffic, inst = read_profile(tag, path)
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_source": f"{peak_kind} hbm_gbs (burst, kernel timed alone)", "traffic": traffic,
           "algorithmic_bytes_per_launch": int(b_alg), "lookups_per_launch": 0 if path == 7 else lookups,
           "hits_per_launch": hits, "kernel_ms": ms, "profile": f"profiles/{tag}.md" if traffic else None}
    roof = hbm
    if path == 7 and prec in (0, 1) and hits and sm_mhz:
        flops = 2.0 * hits * k
        peak_f = FP64_FMA_PER_SM_CYCLE * 2 * n_sms * sm_mhz * 1e6 / 1e12
        alu = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak_f, "unit": "TFLOP/s",
               "frac": flops / (ms * 1e-3) / 1e12 / peak_f, "traffic": traffic,
               "peak_source": f"FP64 FMA pipe: {FP64_FMA_PER_SM_CYCLE} FMA/SM/cycle x {n_sms} SMs x "
                              f"median SM clock {sm_mhz:.0f} MHz (derived from unit counts; no measured FP64 peak)",
               "flops_per_launch": flops, "flops_definition": "2 x found columns x k (FP64 FMAs of the accumulation)",
               "kernel_ms": ms}
        # the roof the launch is closest to is the one reported; the other beside it
        if alu["frac"] >= hbm["frac"]:
            roof = dict(alu, hbm={k2: v for k2, v in hbm.items() if k2 != "traffic"})
        else:
            roof = dict(hbm, fp64={k2: v for k2, v in alu.items() if k2 != "traffic"})
    if inst is not None and sm_mhz:
        # warp-instruction issue: 4 schedulers per SM, one instruction each per cycle
        peak_issue = n_sms * 4 * sm_mhz * 1e6
        roof["issue"] = {"warp_instructions_per_launch": inst, "achieved_per_s": inst / (ms * 1e-3),
                         "peak_per_s": peak_issue, "frac": inst / (ms * 1e-3) / peak_issue,
                         "peak_source": f"{n_sms} SMs x 4 issue slots x median SM clock {sm_mhz:.0f} MHz"}
    return roof


def build_workload(ctx, name, chem_strings=1500, counts=True):
    """Generate one workload on the host (not timed), load it, and count the
    lookups and hits of its product; returns the state the timings use."""
    import torch
    op, words, desc = make_workload(name, chem_strings)
    t0 = time.perf_counter()
    h = ctx.load_operator(op)
    sub = ctx.build_subspace(op.n_qubits, words)
    ctx.synchronize()
    build_s = time.perf_counter() - t0
    info = h.info()
    D, G = sub.dim, info["n_groups"]
    rng = np.random.default_rng(0)
    dev, s = ctx.device, ctx.stream
    with torch.cuda.stream(s):
        x1 = torch.as_tensor(rng.normal(size=D), device=dev)
        xb = torch.as_tensor(rng.normal(size=(D, 16)), device=dev)
    xs = {(0, 1): x1, (1, 1): x1.float(), (2, 1): x1.float(), (0, 16): xb, (1, 16): xb.float(), (2, 16): xb.float()}
    ys = {key: ctx.empty(tuple(v.shape), v.dtype) for key, v in xs.items()}
    lookups, hits, how = count_lookups(ctx, h, sub, G) if counts else (0, 0, "not counted")
    ctx.synchronize()
    return {"name": name, "op": op, "words": words, "desc": desc, "h": h, "sub": sub, "info": info, "D": D,
            "G": G, "W": sub.W, "elems": D * (G + 1), "xs": xs, "ys": ys, "lookups": lookups, "hits": hits,
            "how": how, "build_s": build_s,
            "n_sms": torch.cuda.get_device_properties(dev).multi_processor_count}


PREC_NAMES = {0: "fp64", 1: "fp32_mixed", 2: "fp32_dot2"}


def time_product(ctx, st, timer, prec, k, steps, warmup):
    x, y = st["xs"][(prec, k)], st["ys"][(prec, k)]
    return timer.time(lambda: ctx.apply_H(st["h"], st["sub"], x, y, prec), steps, warmup)


def product_entry(ctx, st, prec, k, ms, sm_mhz):
    path = ctx.product_path(st["h"], st["sub"], prec, k)
    peak, peak_kind = load_peaks()
    tag = f"apply_H_{st['name']}_{PREC_NAMES[prec]}_k{k}"
    return {"ms": ms, "gelem_s": st["elems"] * k / (ms * 1e-3) / 1e9, "path": PATH_NAMES[path],
            "roofline": roofline_of(ms, path, tag, st["D"], st["W"], k, prec, st["lookups"], st["hits"],
                                    st["info"], peak, peak_kind, sm_mhz, st["n_sms"])}


def measure_head(ctx, st, args, timer, dist, world):
    prec0, k0 = HEAD[st["name"]]
    ms, all_ms = time_product(ctx, st, timer, prec0, k0, args.steps, args.warmup)
    t_max = max_over_ranks(ms, dist, ctx.device)
    return {"ms": ms, "ms_max_over_ranks": t_max, "step_ms_min_max": [float(np.min(all_ms)), float(np.max(all_ms))],
            "value": whole_job_rate(st["elems"] * k0, t_max * 1e-3, world) / 1e9}


def measure_rest(ctx, q, st, args, timer, sm_mhz, head_ms):
    """Every (precision, block width) variant with its roofline, the forced
    scan shapes and half evaluation (spin workloads), and solves."""
    name = st["name"]
    prec0, k0 = HEAD[name]
    variants = {f"{PREC_NAMES[prec0]}_k{k0}": product_entry(ctx, st, prec0, k0, head_ms, sm_mhz)}
    vsteps = max(3, min(args.steps, 10))
    for prec in (0, 1, 2):
        for k in (1, 16):
            if (prec, k) != (prec0, k0):
                ms, _ = time_product(ctx, st, timer, prec, k, vsteps, 3)
                variants[f"{PREC_NAMES[prec]}_k{k}"] = product_entry(ctx, st, prec, k, ms, sm_mhz)
    g = {key: v["gelem_s"] for key, v in variants.items()}
    variants["mixed_k16_over_fp64_k1"] = g["fp32_mixed_k16"] / g["fp64_k1"]
    variants["mixed_k16_over_fp64_k16"] = g["fp32_mixed_k16"] / g["fp64_k16"]
    variants["dot2_k16_over_fp64_k1"] = g["fp32_dot2_k16"] / g["fp64_k1"]
    variants["fp64_k16_over_fp64_k1"] = g["fp64_k16"] / g["fp64_k1"]
    info = st["info"]
    if name != "chem" and st["W"] <= 4:
        # every group-scan launch shape, forced (the tuner picks among these),
        # and the half evaluation (lower-triangle groups by MSOB, mirrored by
        # FP64 atomic adds; summation order varies between runs)
        for mode, tagm in ((1, "scan"), (3, "half")):
            if mode == 3 and not (info["is_hermitian"] and info["is_real"]):
                continue
            ctx.set_tuning(1, mode)
            for lanes, order, tag in ((1, 1, "lanes1"), (8, 1, "lanes8"), (1, 2, "hash_order")):
                ctx.set_tuning(2, lanes)
                ctx.set_tuning(5, order)
                for prec, k in ((0, 1), (0, 16)) if mode == 3 else ((0, 1), (1, 16)):
                    ms, _ = time_product(ctx, st, timer, prec, k, vsteps, 3)
                    variants[f"{PREC_NAMES[prec]}_k{k}_{tagm}_{tag}"] = {
                        "ms": ms, "gelem_s": st["elems"] * k / (ms * 1e-3) / 1e9}
            ctx.set_tuning(1, 0)
            ctx.set_tuning(2, 0)
            ctx.set_tuning(5, 0)
    # one full ground-state solve per precision (not part of the timed steps):
    # the first call on the pair ("seconds": basis allocation and graph
    # capture included) and the same solve again ("warm_seconds")
    solve = {}
    if not args.no_solve:
        for pname, prec in (("fp64", 0), ("fp32_mixed", 1), ("fp32_dot2", 2)):
            times = []
            for _ in range(2):
                ctx.synchronize()
                t0 = time.perf_counter()
                e, inf = ctx.lanczos_ground_state(st["h"], st["sub"], check=False, precision=prec,
                                                  max_steps=args.solve_steps, tol=1e-9)
                ctx.synchronize()
                times.append(time.perf_counter() - t0)
            solve[pname] = {"seconds": times[0], "warm_seconds": times[1], "energy": e, "steps": inf["steps"],
                            "applies": inf["applies"], "residual": inf["residual"],
                            "status": q.STATUS.get(inf["status"], inf["status"])}
        solve["product_ms_fp64_k1"] = variants["fp64_k1"]["ms"]
        solve["fp64"]["over_products"] = solve_over_products(solve["fp64"], solve["product_ms_fp64_k1"])
    return variants, solve


def solve_over_products(entry, product_ms):
    """Warm solve time over the time of its products (applies x the timed
    FP64 single-vector product): the eigensolver's overhead around H_S x."""
    if not product_ms or not entry.get("applies"):
        return None
    return entry["warm_seconds"] * 1e3 / (entry["applies"] * product_ms)


def workload_summary(st):
    return {"workload": st["name"], "description": st["desc"], "dim": st["D"], "groups": st["G"],
            "qubits": st["op"].n_qubits, "terms": st["info"]["n_terms_in"], "build_s": st["build_s"],
            "counts": {"lookups_per_vector": st["lookups"], "hits_per_vector": st["hits"], "how": st["how"]}}


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
    ctx = q.create(local)
    for knob, value in PATH_KNOBS[args.path]:
        ctx.set_tuning(knob, value)
    timer = Timer(ctx, dist)
    name = args.workload
    prec0, k0 = HEAD[name]
    st = build_workload(ctx, name, args.chem_strings, counts=not args.skip_counts)
    # clocks are sampled over the headline's timed steps
    with ClockSampler(local) as clk:
        head = measure_head(ctx, st, args, timer, dist, world)
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] if clocks else None
    head_entry = product_entry(ctx, st, prec0, k0, head["ms"], sm_mhz)
    h, sub, op, words = st["h"], st["sub"], st["op"], st["words"]
    variants = solve = None
    if not args.product_only:
        variants, solve = measure_rest(ctx, q, st, args, timer, sm_mhz, head["ms"])

    # end to end through the host-buffer ABI call (pinned host memory)
    hx = st["xs"][(prec0, k0)]
    hdt = torch.float64 if prec0 == 0 else torch.float32
    xh = torch.empty(tuple(hx.shape), dtype=hdt, pin_memory=True).numpy()
    xh[:] = hx.cpu().numpy()
    yh = torch.empty(tuple(hx.shape), dtype=hdt, pin_memory=True).numpy()
    for _ in range(args.warmup):
        ctx.apply_H_host(h, sub, xh, prec0, out=yh)
    et = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ctx.apply_H_host(h, sub, xh, prec0, out=yh)
        et.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(et)), dist, ctx.device)
    e2e = {"value": whole_job_rate(st["elems"] * k0, e2e_s, world) / 1e9, "unit": "Gelem/s",
           "h2d_bytes_per_step": int(xh.nbytes), "d2h_bytes_per_step": int(yh.nbytes), "ms_per_step": e2e_s * 1e3,
           "call": "qsd_apply_H_host (pinned host x and y, copies inside the call)"}
    del xh, yh
    for key in list(st["ys"]):
        if key != (prec0, k0):
            del st["ys"][key]

    extra = {}
    if not args.product_only and not args.no_extra and name == "chem":
        for other in SPIN_EXTRAS:
            ost = build_workload(ctx, other)
            o = workload_summary(ost)
            ohead = measure_head(ctx, ost, args, timer, dist, world)
            o["value"] = ohead["value"]
            o["variants"], o["solve"] = measure_rest(ctx, q, ost, args, timer, sm_mhz, ohead["ms"])
            oh, osub, oop = ost["h"], ost["sub"], ost["op"]
            if not args.no_csr:
                o["csr_build"] = run_csr(ctx, oh, osub)
            if not args.no_solve:
                o["lobpcg_k4"] = run_lobpcg(ctx, oh, osub)
            if not args.no_ramps:
                o["ramps"] = run_ramps(ctx, oh, osub, oop, args.ramps_tau)
            if not args.no_packed:
                o["packed"] = run_packed(ctx, q, oop, other)
            extra[other] = o
            ost.clear()
            osub.free()
            oh.free()

    serve = None
    if not args.product_only and not args.no_serve:
        serve = run_serve(args, q, local)
        if args.serve_compare:
            other = 0 if args.serve_pack_rows else 4096
            serve["compare_pack_rows_%d" % other] = run_serve(args, q, local, pack_rows=other)
        if not args.no_pack_loop:
            serve["packing_closed_loop"] = run_pack_loop(args, q, local)

    cpu = None
    if rank == 0 and not args.no_cpu and not args.product_only:
        cpu = cpu_baseline(op, words, st["G"], k0, target_seconds=args.cpu_seconds)
    if rank == 0:
        summ = workload_summary(st)
        line = {
            "metric": METRIC, "value": head["value"], "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_max_over_ranks"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec0 == 0 else "f32+f64acc",
            "data": "synthetic",
            "config": {"workload": name, "description": st["desc"], "dim": st["D"], "groups": st["G"],
                       "qubits": op.n_qubits, "k": k0,
                       "precision": "fp64" if prec0 == 0 else "fp32 storage, fp64 accumulation",
                       "product_path": head_entry["path"],
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": args.steps, "roofline": head_entry["roofline"], "cpu_baseline": cpu,
            "clocks": clocks, "step_ms_min_max": head["step_ms_min_max"], "counts": summ["counts"],
            "build_s": summ["build_s"], "terms": summ["terms"],
            "variants": variants, "solve": solve, "workloads": extra, "serve": serve,
        }
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_csr(ctx, h, sub):
    """Explicit CSR build: lower triangle by MSOB and mirror, against every
    group of every row (two passes each, device sort of the entries)."""
    csr = {}
    for cname, full in (("msob_lower", False), ("full", True)):
        ts, tc = [], []
        nnz = 0
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
        csr[cname] = {"ms": 1e3 * float(np.mean(ts)), "count_pass_ms": 1e3 * float(np.mean(tc)), "nnz": nnz}
    csr["msob_speedup"] = csr["full"]["ms"] / csr["msob_lower"]["ms"]
    return csr


def run_lobpcg(ctx, h, sub):
    """Block LOBPCG (shifted Jacobi preconditioner, the paper's spiked
    start), 4 lowest eigenpairs, with and without the preconditioner."""
    lob = {}
    for pre in (1, 0):
        ctx.synchronize()
        t0 = time.perf_counter()
        ev, inf = ctx.lobpcg(h, sub, k=4, tol=1e-8, precondition=pre, max_iters=600, check=False)
        ctx.synchronize()
        lob["jacobi" if pre else "none"] = {"seconds": time.perf_counter() - t0, "evals": ev.tolist(),
                                            "iters": inf["iters"], "status": inf["status"],
                                            "max_residual": inf["max_residual"]}
    return lob


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
    """Workloads for the served stream: the three families of the benchmark
    (200-qubit heavy-hex Ising with a fresh seed per request, 6x6 XXZ, and
    the 32-orbital fermionic family with integrals from one of two seeds),
    each with a fresh subspace of log-uniform target dimension.  Host
    generation only (not timed); each request does its own device subspace
    build (sort, dedup, hash, hash order, factored index)."""
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
            n_orb, ne = 32, 8
            key = s_ % 2
            if key not in ferm_ops:
                h1, eri = wl.chem_integrals(n_orb, seed=1000 + key)
                ferm_ops[key] = wl.molecular_qubit_operator(h1, eri)
            op = ferm_ops[key]
            side = int(max(2, round(np.sqrt(target))))
            alpha = wl.excitation_strings(n_orb, ne, side, 4, s_)
            beta = wl.excitation_strings(n_orb, ne, side, 4, s_ + 1)
            words = wl.product_subspace(alpha, beta, n_orb)
        pool.append((fam, op, words))
    # the largest draw is stretched to the top of the range, so that the
    # stream always holds a subspace near the maximum dimension
    big = int(np.argmax([w.shape[0] for _, _, w in pool]))
    fam, op, words = pool[big]
    if fam == "ising":
        words = wl.flip_words(200, int(dmax), 20, seed + 1)
    elif fam == "xxz":
        words = wl.xxz_walk_words(6, 6, int(dmax), 12, seed + 1)
    else:
        side = int(np.sqrt(dmax))
        words = wl.product_subspace(wl.excitation_strings(32, 8, side, 4, seed + 1),
                                    wl.excitation_strings(32, 8, side, 4, seed + 2), 32)
    pool[big] = (fam, op, words)
    return pool


def run_pack_loop(args, q, local, slots=64, n_requests=512):
    """Where packing pays: the solver alone in closed loop (operators loaded
    and subspaces built beforehand; 512 requests submitted at once into 64
    slots), with packing on (every request) and off, for subspaces of
    1e3-4e3 rows and of 1e3-3e4 rows of the three served families."""
    import torch
    ctx = q.create(local)
    params = dict(precision=q.QSD_FP32_DOT2, max_steps=300, tol=1e-7, check_every=10)
    out = {"slots": slots, "requests": n_requests, "precision": "fp32_dot2 + fp64 refinement",
           "note": "closed loop, solver only: subspaces built and operators loaded before the timed "
                   "region; each configuration warmed by one pass over the pool"}
    loaded = {}
    for dmax in (4e3, 3e4):
        pool = serve_pool(args.serve_pool, args.serve_seed, 1e3, dmax)
        items = []
        for fam, op, words in pool:
            if id(op) not in loaded:
                loaded[id(op)] = ctx.load_operator(op)
            items.append((loaded[id(op)], ctx.build_subspace(op.n_qubits, words)))
        ctx.synchronize()
        order = np.random.default_rng(args.serve_seed).integers(0, len(items), size=n_requests).tolist()
        res = {}
        for rows in (0, 1 << 20):
            with q.Server(ctx, budget_bytes=64 << 30, max_active=slots) as srv:
                srv.set_pack_rows(rows)
                for t in [srv.submit(h, s_, **params) for h, s_ in items]:
                    srv.wait(t)
                t0 = time.perf_counter()
                tickets = [srv.submit(items[i][0], items[i][1], **params) for i in order]
                rr = [srv.wait(t) for t in tickets]
                wall = time.perf_counter() - t0
                st = srv.stats()
            lat = np.array([r["t_done"] - r["t_submit"] for r in rr]) * 1e3
            res["packed" if rows else "unpacked"] = {
                "solves_per_s": n_requests / wall, "ok": sum(r["status"] == "OK" for r in rr),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "packed_chunks": st["packed_chunks"]}
        res["packed_over_unpacked"] = res["packed"]["solves_per_s"] / res["unpacked"]["solves_per_s"]
        out["rows_1e3_%de3" % int(dmax / 1e3)] = res
        for _, sub in items:
            sub.free()
    for h in loaded.values():
        h.free()
    ctx.close()
    return out


def run_serve(args, q, local, pack_rows=None, dmin=1e3, dmax=2e6, slots=None, n_requests=None):
    """Poisson arrivals (512 by default) at 0.8x the measured closed-loop
    capacity; latency from arrival to energy ready, including the request's
    device build."""
    import torch
    pack_rows = args.serve_pack_rows if pack_rows is None else pack_rows
    slots = args.serve_slots if slots is None else slots
    rng = np.random.default_rng(args.serve_seed)
    pool = serve_pool(args.serve_pool, args.serve_seed, dmin, dmax)
    client = q.create(local)
    srvctx = q.create(local)
    budget = int(args.serve_budget_gb * (1 << 30))
    params = dict(precision=q.QSD_FP32_DOT2, max_steps=300, tol=1e-7, check_every=10)
    handles = []
    loaded = {}  # each distinct Hamiltonian is loaded (grouped) once and stays resident

    def build(i):
        fam, op, words = pool[i]
        if id(op) not in loaded:
            loaded[id(op)] = client.load_operator(op)
        h = loaded[id(op)]
        sub = client.build_subspace(op.n_qubits, words)
        handles.append(sub)
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

    with q.Server(srvctx, budget_bytes=budget, max_active=slots) as srv:
        srv.set_pack_rows(pack_rows)
        host_t0 = time.perf_counter()
        # closed-loop capacity: every pool item submitted at once
        burst, t_burst = run(list(range(len(pool))), [0.0] * len(pool), srv, host_t0)
        capacity = len(pool) / t_burst
        lam = 0.8 * capacity
        n = args.serve_requests if n_requests is None else n_requests
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
           "max_active": slots, "budget_bytes": budget, "peak_bytes": st["peak_bytes"],
           "per_family_p50_ms": {k: float(np.percentile(v, 50)) for k, v in fams.items()},
           "phases": phases, "pack_rows": pack_rows,
           "packed_requests": st["packed_requests"], "packed_chunks": st["packed_chunks"],
           "candidate_dims_min_max": [int(min(dims)), int(max(dims))],
           "precision": "fp32_dot2 + fp64 refinement", "tol": params["tol"],
           "families": {"ising": "200-qubit heavy-hex, fresh seed per pool entry",
                        "xxz": "6x6 periodic", "fermion": "32 orbitals, integrals from seed 1000 or 1001"},
           "note": "latency = arrival to energy ready, including the request's device subspace build "
                   "(and the operator's load and grouping the first time a Hamiltonian is seen; "
                   "loaded Hamiltonians stay resident); host synthetic generation excluded "
                   "(pool of %d workloads)" % len(pool)}
    client.close()
    srvctx.close()
    return out


# ------------------------------------------------------------------ CPU arm
def cpu_baseline(op, words, G, k=1, target_seconds=12.0, sample_rows=None):
    """The plain oracle product of k vectors on a bounded sample of rows,
    timed on the host cores; returns Gelem/s on the same count
    (rows * (groups + 1) * k)."""
    import oracle
    keys = oracle.sort_unique(words)
    D = keys.shape[0]
    x = np.random.default_rng(0).normal(size=(D, k) if k > 1 else D)
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
    return {"value": sample_rows * (G + 1) * k / dt / 1e9, "unit": "Gelem/s",
            "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle", "seconds": dt,
            "sample": f"{sample_rows} of {D} rows (uniform sample), FP64 product of {k} vector(s), OpenMP over rows"}


def run_reference(args):
    """The CPU oracle on the host cores, on the GPU arm's workload, metric and
    unit: each step one bounded uniform sample of rows of the headline
    product (same precision and block width)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    op, words, desc = make_workload(args.workload, args.chem_strings)
    prec0, k0 = HEAD[args.workload]
    keys = oracle.sort_unique(words)
    # group count by the oracle's own definition (distinct flip sets)
    G = oracle.groups(op).shape[0]
    D = keys.shape[0]
    x = np.random.default_rng(0).normal(size=(D, k0) if k0 > 1 else D)
    rng = np.random.default_rng(2)
    probe = np.sort(rng.choice(D, size=min(D, 256), replace=False))
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
    value = n * (G + 1) * k0 / (ms * 1e-3) / 1e9
    cores = int(os.environ["OMP_NUM_THREADS"])
    sample = f"{n} of {D} rows per step (uniform sample), FP64 product of {k0} vector(s), OpenMP over rows"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "dim": D, "groups": G, "k": k0,
                   "precision": "fp64", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="chem", choices=["chem", "xxz", "tfim", "ising"])
    ap.add_argument("--product-only", action="store_true",
                    help="time the headline product steps (and the host-buffer call) only")
    ap.add_argument("--no-extra", action="store_true", help="skip the Ising and XXZ workloads")
    ap.add_argument("--chem-strings", type=int, default=1500,
                    help="alpha and beta strings of the fermionic workload (reduced cases for profiling)")
    ap.add_argument("--path", default="auto", choices=sorted(PATH_KNOBS),
                    help="force a product path (profiling); auto lets the library choose")
    ap.add_argument("--skip-counts", action="store_true",
                    help="do not count lookups and hits (the roofline's byte count is then incomplete)")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--solve-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-step-seconds", type=float, default=2.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-csr", action="store_true", help="skip the CSR build timing")
    ap.add_argument("--no-packed", action="store_true", help="skip the packed-launch timing")
    ap.add_argument("--no-ramps", action="store_true", help="skip the RAMPS timing")
    ap.add_argument("--ramps-tau", type=float, default=1e-7)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-pool", type=int, default=36)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-pack-rows", type=int, default=4096,
                    help="requests up to this many rows run in packed chunks (0: never)")
    ap.add_argument("--no-pack-loop", action="store_true",
                    help="skip the closed-loop packing comparison")
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
