#!/usr/bin/env python3
"""Benchmark of the hot path: rank-by-degree orientation + vertex-centric
hashed triangle counting, on the random-geometric-graph workload (2^22 points
uniform in the unit square, radius set for mean degree 64, seed 2).

One step = one tc_count_async over the device-resident CSR: degree,
orientation counts, scan, compaction, binning, hash build + probe, 64-bit
reduction. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun) every rank holds the whole CSR and counts the
vertices u with u % N == rank (the workload partition of Sec. 5.1); the
per-rank counts are summed once, after timing. The reference arm times the
CPU oracle on the host cores (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(name="rgg-2^22-meandeg64-seed2", points_log2=22, mean_degree=64.0, seed=2)
REF_SAMPLE = dict(name="rgg-2^20-meandeg64-seed2", points_log2=20, mean_degree=64.0, seed=2)
# --workload: the other single-graph configurations, measured the same way
OTHER_WORKLOADS = {
    "rmat16": dict(name="rmat-s16-ef16-seed1", graph="rmat16"),
    "rmat22": dict(name="rmat-s22-ef16-seed1", graph="rmat22"),
    "rmat26": dict(name="rmat-s26-ef16-seed3", graph="rmat26"),
}
METRIC = "triangle-count TEPS"
UNIT = "edges/s"
FALLBACK_HBM_GBS = 6800.0
PROFILE = os.path.join(ROOT, "profiles", "k_count_pack__rgg22.md")
COUNT_SRC = os.path.join(ROOT, "paper_2103_08053_gb300", "csrc", "count.cu")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def make_graph(spec):
    import graphgen as G
    if "graph" in spec:
        return G.workload(spec["graph"])
    return G.rgg(1 << spec["points_log2"], spec["mean_degree"], seed=spec["seed"])


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- roofline

def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(p))["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def count_source_hash() -> str:
    return hashlib.sha256(open(COUNT_SRC, "rb").read()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the counting kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    h = re.search(r"count\.cu sha256\[:16\]:\s*([0-9a-f]{16})", text)
    b = re.search(r"dram bytes per launch \(read\+write\):\s*([0-9.eE+]+)", text)
    if not h or not b or h.group(1) != count_source_hash():
        return None
    return float(b.group(1))


def count_phase_bytes(n: int, m: int, wplus: int) -> int:
    """Algorithmic bytes of one counting pass: dag_ptr of every u (4(n+1)),
    each out-list read once to build its table (4m), the bounds of N+(v) for
    every out-edge (8m) and every probed 2-hop key (4 W+)."""
    return 4 * (n + 1) + 4 * m + 8 * m + 4 * wplus


# ------------------------------------------------- batched and served graphs

BATCH = dict(name="batch-4096-seed4", graphs=4096, seed=4)
SERVE = dict(rate=2000.0, pool=256, pool_seed=5, big_fraction=0.01, big_scale=22, budget_gb=40, seed=5)


def measure_batched(T, torch, dev, steps: int):
    """tc_count_batch over the 4096-graph batch (CUDA-graph replay) against a
    loop of tc_count over the same graphs, on the same GPU."""
    import numpy as np

    import graphgen as G
    t0 = time.time()
    gs = G.batch(BATCH["seed"], BATCH["graphs"])
    gen_s = time.time() - t0
    tensors = [(g.n, torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev),
                torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(dev)) for g in gs]
    edges = sum(g.m for g in gs)
    with T.Context(dev.index) as c:
        t = time.time()
        # the tuner's on-disk cache lives in the system's temporary directory
        tuned = c.autotune(tensors, cache_path=os.path.join(tempfile.gettempdir(), "trust_gb300_tune_cache.txt"))
        tune_s = time.time() - t
        counts = c.count_batch(tensors)  # first call captures the CUDA graph
        c.count_batch(tensors)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for _ in range(steps):
            c.count_batch(tensors)
        batch_s = (time.perf_counter() - t) / steps
        loop = [c.count(n, rp, col) for n, rp, col in tensors[:64]]  # warm-up
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        loop = [c.count(n, rp, col) for n, rp, col in tensors]
        loop_s = time.perf_counter() - t
    import oracle
    sample = list(range(0, BATCH["graphs"], BATCH["graphs"] // 32))
    want = [oracle.count(gs[i]) for i in sample]
    return {
        "workload": BATCH["name"], "graphs": len(gs), "edges": edges, "generation_s": round(gen_s, 1),
        "ms_per_batch": batch_s * 1e3, "graphs_per_s": len(gs) / batch_s, "edges_per_s": edges / batch_s,
        "loop_graphs_per_s": len(gs) / loop_s, "speedup_vs_loop": loop_s / batch_s, "steps": steps,
        "autotuned": {k: tuned[k] for k in ("warp_max_out_degree", "warp_area_ints", "warp_min_buckets", "chunk",
                                             "warps_per_block", "item_neighbors")}, "tune_s": round(tune_s, 1),
        "parity": {"batch_equals_loop": counts == loop,
                   "oracle_sample": len(sample), "oracle_equal": [counts[i] for i in sample] == want},
    }


def measure_serving(T, torch, dev, seconds: float):
    """Poisson arrivals (rate 2000/s) of requests drawn from the batched
    distribution, 1% R-MAT scale-22 graphs, admitted under a 40 GB budget;
    submit -> poll-ready latency and completed graphs/s."""
    import numpy as np

    import graphgen as G
    pool = G.batch(SERVE["pool_seed"], SERVE["pool"])
    big = [G.rmat(SERVE["big_scale"], 16, seed=SERVE["seed"] + i) for i in range(2)]
    graphs = pool + big
    pinned = []
    for g in graphs:
        rp = torch.from_numpy(g.row_ptr.astype(np.int32)).pin_memory()
        col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).pin_memory()
        pinned.append((g.n, rp, col, rp.numpy(), col.numpy()))
    with T.Context(dev.index) as c:  # every graph counted alone first
        alone = [c.count(n, rp.to(dev), col.to(dev)) for n, rp, col, _, _ in pinned]
    rng = np.random.default_rng(SERVE["seed"])
    n_req = max(1, int(SERVE["rate"] * seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / SERVE["rate"], n_req))
    pick = np.where(rng.random(n_req) < SERVE["big_fraction"], len(pool) + rng.integers(0, len(big), n_req),
                    rng.integers(0, len(pool), n_req))
    with T.Context(dev.index, mem_budget=SERVE["budget_gb"] << 30) as c:
        warm = c.submit_borrowed(pinned[0][0], pinned[0][3], pinned[0][4])  # starts the serving worker
        c.drain()
        assert c.poll(warm) == alone[0]
        submit_t = np.zeros(n_req)
        done_t = np.zeros(n_req)
        result = [None] * n_req
        outstanding = {}
        nxt = 0
        t0 = time.perf_counter()
        while nxt < n_req or outstanding:
            now = time.perf_counter() - t0
            while nxt < n_req and arrivals[nxt] <= now:
                n, _, _, rp_np, col_np = pinned[pick[nxt]]
                outstanding[c.submit_borrowed(n, rp_np, col_np)] = nxt
                submit_t[nxt] = time.perf_counter() - t0
                nxt += 1
            for tk in list(outstanding):
                v = c.poll(tk)
                if v is not None:
                    i = outstanding.pop(tk)
                    done_t[i] = time.perf_counter() - t0
                    result[i] = v
            if nxt < n_req and not outstanding:
                time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.001)))
    lat = (done_t - submit_t) * 1e3
    edges = sum(graphs[i].m for i in pick)
    span = done_t.max() - submit_t.min()
    return {
        "arrival_rate_per_s": SERVE["rate"], "seconds": seconds, "requests": n_req,
        "big_requests": int((pick >= len(pool)).sum()), "budget_gb": SERVE["budget_gb"],
        "graphs_per_s": n_req / span, "edges_per_s": edges / span,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "identical_to_alone": all(result[i] == alone[pick[i]] for i in range(n_req)),
        "submission": "tc_submit_borrowed from pinned host memory",
    }


def time_count(ctx, torch, dev, n, rp, col, reps=10):
    """Median ms of tc_count_async (orientation + counting) by CUDA events."""
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        ctx.count_async(n, rp, col, out, err, stream=stream)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.count_async(n, rp, col, out, err, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    if int(err.item()) != 0:
        raise SystemExit("counting failed during a study")
    return statistics.median(ts), int(out.item())


def measure_reorder(T, torch, dev, graphs):
    """Sec. 4.1 study: for each graph, tc_reorder by in-degree and by
    collective out-degree; the max collision and Eq. 2 cost of 32-bucket
    tables (x mod 32 and multiplicative), and the counting time under both
    table hashes with the warp workers in vertex order (as the paper's queue
    hands them out), and with the library's defaults (the ordered warp list
    on graphs of >= 2^24 entries), before and after reordering. The count
    must not change."""
    rows = []
    for name, (n, rp, col) in graphs.items():
        with T.Context(dev.index) as c:
            variants = [("none", rp, col, 0.0)]
            for kind, label in ((T.TC_REORDER_INDEGREE, "indegree"), (T.TC_REORDER_COLLECTIVE, "collective")):
                c.reorder(n, rp, col, kind, relabel=True)  # warm-up
                torch.cuda.synchronize(dev)
                t = time.perf_counter()
                _, rp2, col2 = c.reorder(n, rp, col, kind, relabel=True)
                variants.append((label, rp2, col2, (time.perf_counter() - t) * 1e3))
            base = None
            for label, r, cc, ms_re in variants:
                d = c.orient(n, r, cc)
                st = c.dag_stats(d)
                d.free()
                row = {"graph": name, "order": label, "reorder_ms": ms_re,
                       "max_collision_mod32": st["max_collision_mod32"], "phi_mod32": st["phi_mod32"],
                       "max_collision_mult32": st["max_collision_mult32"], "phi_mult32": st["phi_mult32"]}
                for prm, key in ((dict(warp_order=2), "count_ms_mult_hash"),
                                 (dict(warp_order=2, hash_mode=1), "count_ms_mod_hash"),
                                 ({}, "count_ms_defaults")):
                    with T.Context(dev.index, params=prm) as ch:
                        ms, tri = time_count(ch, torch, dev, n, r, cc)
                    row[key] = ms
                    base = tri if base is None else base
                    row["count_equal"] = tri == base
                rows.append(row)
                if label != "none":
                    del r, cc
    return rows


def measure_ablation(T, torch, dev, graphs):
    """Sec. 3.3 and Sec. 4.2 ablations on the given graphs. Sec. 3.3: the
    worker cycles spent building tables vs probing them, vertex-centric
    Algorithm 1 vs the edge-centric Algorithm 2 (N+(u)'s table rebuilt for
    every out-edge). Sec. 4.2: how the warp workers spread the 2-hop lists
    over their lanes -- virtual combination (the design, with 16-byte or
    one-key loads) vs warp-centric, subwarps of 8 and 16 lanes and physical
    combination. count_ms is timed without the cycle counters; the count must
    be the same in every mode."""
    modes = [("vertex-centric, VC, 16- or 32-byte loads (default)", {}),
             ("vertex-centric, VC, scalar loads", dict(scalar_loads=1)),
             ("vertex-centric, warp-centric (WC)", dict(balance=T.TC_BALANCE_WC)),
             ("vertex-centric, subwarp 8 (SW8)", dict(balance=T.TC_BALANCE_SW8)),
             ("vertex-centric, subwarp 16 (SW16)", dict(balance=T.TC_BALANCE_SW16)),
             ("vertex-centric, physical combination (PC)", dict(balance=T.TC_BALANCE_PC)),
             ("edge-centric (Algorithm 2)", dict(edge_centric=1))]
    rows = []
    for name, (n, rp, col) in graphs.items():
        base = None
        for label, prm in modes:
            with T.Context(dev.index, params=dict(prm, record_timing=2)) as c:
                tri = c.count(n, rp, col)          # blocking: reads the cycle counters back
                t = c.read_timing()
            with T.Context(dev.index, params=prm) as c:
                ms, tri2 = time_count(c, torch, dev, n, rp, col, reps=5)
            base = tri if base is None else base
            cyc = t["build_cycles"] + t["probe_cycles"]
            rows.append({"graph": name, "mode": label, "count_ms": ms,
                         "build_share": t["build_cycles"] / cyc if cyc else None,
                         "count_equal": tri == base == tri2})
    return rows


def reorder_profile_run(args):
    """The launch sequence for profiling Sec. 4.1's reorderings with ncu: one
    graph, and for each order (none, in-degree, collective out-degree) one
    tc_count with the warp workers in vertex order, so that k_count_pack runs
    exactly three times, in that order. Prints one JSON line describing them
    (an ncu run over this command captures the counters: shared-load
    instructions, their bank conflicts, the L2 hit rate)."""
    import numpy as np
    import torch

    import graphgen as G
    import paper_2103_08053_gb300 as T
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g = G.workload(args.reorder_profile)
    n = g.n
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(dev)
    rows = []
    with T.Context(0, params=dict(warp_order=2, hash_mode=args.profile_hash_mode)) as c:
        for kind, label in ((None, "none"), (T.TC_REORDER_INDEGREE, "indegree"),
                            (T.TC_REORDER_COLLECTIVE, "collective")):
            r, cc = (rp, col) if kind is None else c.reorder(n, rp, col, kind, relabel=True)[1:]
            d = c.orient(n, r, cc)
            st = c.dag_stats(d)
            d.free()
            rows.append({"order": label, "triangles": c.count(n, r, cc),
                         "max_collision_mod32": st["max_collision_mod32"],
                         "max_collision_mult32": st["max_collision_mult32"]})
    print(json.dumps({"reorder_profile": args.reorder_profile, "hash_mode": args.profile_hash_mode, "n": n, "m": g.m,
                      "k_count_pack_launches": [r["order"] for r in rows], "rows": rows}), flush=True)


# -------------------------------------------------------------- the arms

def run_gb300(args):
    import numpy as np
    import torch

    import paper_2103_08053_gb300 as T

    rank, local_rank, world = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

    t0 = time.time()
    g = make_graph(WORKLOAD)
    log(f"[rank {rank}] generated {WORKLOAD['name']}: n={g.n} m={g.m} in {time.time() - t0:.1f}s")
    bits = 32 if g.nnz < 2 ** 31 else 64
    rp_h = g.row_ptr.astype(np.int32 if bits == 32 else np.int64)
    col_h = np.ascontiguousarray(g.col, dtype=np.int32)
    rp = torch.from_numpy(rp_h).to(dev)
    col = torch.from_numpy(col_h).to(dev)
    from paper_2103_08053_gb300 import shard
    params = dict(record_timing=1, **shard.shard_params(rank, world))
    ctx = T.Context(local_rank, params=params)
    stream = torch.cuda.current_stream(dev)

    # exact statistics of the DAG (outside the timed region): W+ for the byte model
    full = T.Context(local_rank)
    dag = full.orient(g.n, rp, col)
    st = full.dag_stats(dag)
    dag.free()
    full.close()

    out = torch.zeros(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        ctx.count_async(g.n, rp, col, out, err, stream=stream)
    torch.cuda.synchronize(dev)
    my_count = int(out.item())
    if int(err.item()) != 0:
        raise SystemExit(f"counting failed with status {int(err.item())}")
    ctx.read_timing()  # drop warm-up timings
    launches0 = ctx.kernel_launches()

    sampler = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.count_async(g.n, rp, col, out, err, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = e0.elapsed_time(e1)
    launches = ctx.kernel_launches() - launches0
    tm = ctx.read_timing()
    total_count, elapsed_ms = shard.combine(my_count, elapsed_ms, device=dev)
    ms_per_step = elapsed_ms / args.steps
    value = g.m / (ms_per_step / 1e3)

    # end to end through the C ABI from pinned host memory: H2D of the CSR, the
    # whole path, D2H of the count, every step
    rp_pin = torch.from_numpy(rp_h).pin_memory()
    col_pin = torch.from_numpy(col_h).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(max(3, args.warmup)):
        ctx.count_host(g.n, rp_pin.numpy(), col_pin.numpy(), stream=stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    # each call blocks until its count is on the host: time every step, report
    # the median (one host-side stall would otherwise move the mean) and the mean
    e2e_each = []
    t_e = time.perf_counter()
    for _ in range(e2e_steps):
        t_s = time.perf_counter()
        e2e_count = ctx.count_host(g.n, rp_pin.numpy(), col_pin.numpy(), stream=stream)
        e2e_each.append((time.perf_counter() - t_s) * 1e3)
    torch.cuda.synchronize(dev)
    e2e_mean_ms = (time.perf_counter() - t_e) * 1e3 / e2e_steps
    e2e_ms = statistics.median(e2e_each)
    _, e2e_ms = shard.combine(0, e2e_ms, device=dev)
    # the host-to-device copy alone on this machine (context for the end-to-end number)
    rp_d = torch.empty_like(rp_pin, device=dev)
    col_d = torch.empty_like(col_pin, device=dev)
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(3):
        rp_d.copy_(rp_pin, non_blocking=True)
        col_d.copy_(col_pin, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize(dev)
    h2d_ms = h0.elapsed_time(h1) / 3
    del rp_d, col_d
    ctx.read_timing()
    ctx.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_src = measured_hbm_peak()
    count_ms = tm["count_ms"] / max(tm["calls"], 1)
    bytes_count = count_phase_bytes(g.n, g.m, st["wedges_plus"])
    achieved = bytes_count / (count_ms / 1e3) / 1e9
    traffic = profiled_traffic() if WORKLOAD["name"] == "rgg-2^22-meandeg64-seed2" else None

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD["name"], "n": g.n, "m": g.m, "nnz": g.nnz, "offset_bits": bits,
            "triangles": total_count, "wedges_plus": st["wedges_plus"], "max_out_degree": st["max_out_degree"],
            "bins": {"skip": st["n_skip"], "warp": st["n_warp"], "block": st["n_block"]},
            "step": "tc_count_async: orientation + binning + hash build/probe + reduction, CSR resident in HBM",
            "l2": "no flush: inputs larger than L2 (col %.2f GB, DAG %.2f GB vs 129 MB)"
                  % (g.nnz * 4 / 1e9, (g.m + g.n) * 4 / 1e9),
            "parallelism": f"workload partition u % {world}" if world > 1 else "single GPU",
        },
        "phases_ms": {"orient": tm["orient_ms"] / max(tm["calls"], 1), "bin": tm["bin_ms"] / max(tm["calls"], 1),
                      "count": count_ms},
        "roofline": {"kernel": "counting kernels (k_count_block + k_count_pack)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                     else "fallback 6.8 TB/s", "traffic": traffic,
                     "algorithmic_bytes_per_launch": bytes_count,
                     "bytes_model": "4(n+1) + 12m + 4W+"},
        "e2e": {"value": g.m / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "stat": f"median of {e2e_steps} timed calls", "mean_ms_per_step": e2e_mean_ms,
                "max_ms_per_step": max(e2e_each),
                "h2d_bytes_per_step": int(rp_h.nbytes + col_h.nbytes), "d2h_bytes_per_step": 16,
                "h2d_copy_ms": h2d_ms, "host_pinned": bool(col_pin.is_pinned()),
                "count_equal_device": e2e_count == my_count,
                "api": "tc_count_host (pinned host CSR)"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # the batched, served and study sections and the CPU baseline are
    # single-GPU measurements: a multi-rank run reports the sharded step only
    single = world == 1
    if args.batched and single:
        result["batched"] = measure_batched(T, torch, dev, steps=args.batch_steps)
    if args.serve_seconds > 0 and single:
        result["serving"] = measure_serving(T, torch, dev, args.serve_seconds)
    if args.reorder and single:
        import numpy as np

        import graphgen as G
        big = G.rmat(22, 16, seed=5)
        gs = {WORKLOAD["name"]: (g.n, rp, col),
              "rmat-s22-ef16-seed5": (big.n, torch.from_numpy(big.row_ptr.astype(np.int32)).to(dev),
                                      torch.from_numpy(np.ascontiguousarray(big.col, dtype=np.int32)).to(dev))}
        result["reorder_study"] = measure_reorder(T, torch, dev, gs)
    if args.ablation and single:
        import numpy as np

        import graphgen as G
        small = G.workload("rmat16")
        gs = {WORKLOAD["name"]: (g.n, rp, col),
              "rmat-s16-ef16-seed1": (small.n, torch.from_numpy(small.row_ptr.astype(np.int32)).to(dev),
                                      torch.from_numpy(np.ascontiguousarray(small.col, dtype=np.int32)).to(dev))}
        result["ablation_study"] = measure_ablation(T, torch, dev, gs)
    if not args.no_cpu_baseline and single:
        import oracle
        cores = oracle.max_threads()
        t = time.perf_counter()
        want = oracle.count(g, threads=cores)
        cpu_s = time.perf_counter() - t
        result["cpu_baseline"] = {"value": g.m / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"one oracle orientation + node-iterator count of the whole "
                                            f"{WORKLOAD['name']} graph ({cpu_s:.1f} s)"}
        result["parity"] = {"oracle": want, "gpu": total_count, "equal": want == total_count}
    if dist:
        dist.destroy_process_group()
    print(json.dumps(result), flush=True)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return  # the CPU oracle runs once, on rank 0
    import oracle
    g = make_graph(REF_SAMPLE)
    # rank 0 alone does the work: all host cores, whatever OMP_NUM_THREADS
    # the launcher set for its ranks
    cores = max(oracle.max_threads(), len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                else (os.cpu_count() or 1))
    for _ in range(args.warmup):
        oracle.count(g, threads=cores)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.count(g, threads=cores)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = g.m / (ms / 1e3)
    sample = (f"one oracle orientation + node-iterator count per step of {REF_SAMPLE['name']} "
              f"(same family as {WORKLOAD['name']}, 1/4 of its points), {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "sample": REF_SAMPLE["name"], "n": g.n, "m": g.m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=1, help="1: also time the 4096-graph batch (rank 0)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--workload", choices=["rgg22", *OTHER_WORKLOADS], default="rgg22",
                    help="graph of the timed steps (default: the RGG 2^22 benchmark graph); the batched, serving "
                         "and study sections always use their own workloads")
    ap.add_argument("--ablation", type=int, default=1,
                    help="1: also run the Sec. 3.3 (build/probe, edge-centric) and Sec. 4.2 (WC/SW/PC/VC) ablations (rank 0)")
    ap.add_argument("--reorder", type=int, default=1,
                    help="1: also run the Sec. 4.1 reordering study (rank 0)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="seconds of Poisson arrivals for the serving measurement (0: skip; the config is 60)")
    ap.add_argument("--reorder-profile", default=None, metavar="GRAPH",
                    help="only run the Sec. 4.1 profiling sequence on this workload (e.g. rgg20, rmat21) and exit")
    ap.add_argument("--profile-hash-mode", type=int, choices=[0, 1], default=0,
                    help="table hash of the profiling sequence: 0 multiplicative (default), 1 x mod B (Algorithm 1)")
    args = ap.parse_args()
    if args.reorder_profile:
        reorder_profile_run(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload != "rgg22":
        global WORKLOAD
        WORKLOAD = OTHER_WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
