#!/usr/bin/env python3
"""Benchmark of the hot path: rank-by-degree orientation + vertex-centric
hashed triangle counting (Algorithm 1 on N+), on the largest single-GPU
workload: R-MAT scale 26 (67,108,864 vertices, edge factor 16, (a,b,c,d) =
(0.57, 0.19, 0.19, 0.05), seed 3; 1.05 B undirected edges), int32 CSR with
int64 row offsets.

One step = one tc_count_async over the device-resident CSR: degree,
orientation (row-local DAG), binning, hash build + probe, 64-bit reduction.
Prints one JSON line (rank 0) with the main workload's TEPS, and beside it
the random-geometric-graph workload (2^22 points, mean degree 64), the
4096-graph batch, the served Poisson stream and the Sec. 3.3 / 4.1 / 4.2
studies.

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

GOLDEN = os.path.join(ROOT, "tests", "golden")
# single-graph workloads (--workload); the default is the largest one
WORKLOADS = {
    "rmat26": dict(name="rmat-s26-ef16-seed3", graph="rmat26", offset_bits=64, golden="rmat26.json",
                   oracle_fraction=1 / 32, n=1 << 26, nnz_max=2 * 16 << 26),
    "rgg22": dict(name="rgg-2^22-meandeg64-seed2", graph="rgg22", offset_bits=32, oracle_fraction=1.0,
                  n=1 << 22, nnz_max=80 << 22),
    "rmat16": dict(name="rmat-s16-ef16-seed1", graph="rmat16", offset_bits=32, oracle_fraction=1.0,
                   n=1 << 16, nnz_max=2 * 16 << 16),
    "rmat22": dict(name="rmat-s22-ef16-seed1", graph="rmat22", offset_bits=32, oracle_fraction=1.0,
                   n=1 << 22, nnz_max=2 * 16 << 22),
}
DEFAULT_WORKLOAD = "rmat26"
# the reference arm's per-step sample of the main workload's vertices
REF_FRACTION = 1 / 256
METRIC = "triangle-count TEPS"
UNIT = "edges/s"
FALLBACK_HBM_GBS = 6800.0
COUNT_SRC = os.path.join(ROOT, "paper_2103_08053_gb300", "csrc", "count.cu")
# ncu summaries with the DRAM bytes of one counting step, per workload
PROFILES = {"rgg22": os.path.join(ROOT, "profiles", "k_count_pack__rgg22.md"),
            "rmat26": os.path.join(ROOT, "profiles", "counting__rmat26.md")}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def make_graph(spec):
    import graphgen as G
    return G.workload(spec["graph"])


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


def profiled_traffic(key: str):
    """DRAM bytes of the counting kernels per step from the committed ncu
    summary of workload `key`, or None when there is none or the kernel
    source changed since the capture."""
    try:
        text = open(PROFILES[key]).read()
    except (OSError, KeyError):
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
SERVE = dict(rate=2000.0, big_fraction=0.01, big_scale=22, big_seeds=(5, 6, 7, 8), budget_gb=40, seed=5)


def measure_batched(T, torch, dev, steps: int, gs):
    """tc_count_batch over the 4096-graph batch (CUDA-graph replay) against a
    loop of tc_count over the same graphs, on the same GPU; every graph's
    count against the oracle's."""
    import numpy as np

    import oracle
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
    t = time.time()
    want = oracle.count_many(gs)
    oracle_s = time.time() - t
    return {
        "workload": BATCH["name"], "graphs": len(gs), "edges": edges,
        "ms_per_batch": batch_s * 1e3, "graphs_per_s": len(gs) / batch_s, "edges_per_s": edges / batch_s,
        "loop_graphs_per_s": len(gs) / loop_s, "speedup_vs_loop": loop_s / batch_s, "steps": steps,
        "autotuned": {k: tuned[k] for k in ("warp_max_out_degree", "warp_area_ints", "warp_min_buckets", "chunk",
                                             "warps_per_block", "item_neighbors")}, "tune_s": round(tune_s, 1),
        "parity": {"batch_equals_loop": counts == loop, "oracle_graphs": len(want),
                   "oracle_equal": counts == want, "oracle_s": round(oracle_s, 1)},
    }


def _percentiles(lat_ms):
    import numpy as np
    return {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "mean_ms": float(lat_ms.mean()), "max_ms": float(lat_ms.max())}


def measure_serving(T, torch, dev, seconds: float, pool):
    """Poisson arrivals (rate 2000/s) of triangle-count requests, 99 % drawn
    uniformly from `pool` (independent draws of the batched distribution) and
    1 % R-MAT scale-22 graphs, admitted under a 40 GB budget through
    tc_submit_borrowed; submit -> poll-ready latency and completed graphs/s.
    The same arrival trace is then run through a plain loop of tc_count_host,
    one request after the other, each submitted at its arrival time."""
    import numpy as np

    import graphgen as G
    big = [G.rmat(SERVE["big_scale"], 16, seed=s) for s in SERVE["big_seeds"]]
    graphs = list(pool) + big
    pinned = []
    for g in graphs:
        rp = pinned_copy(torch, g.row_ptr.astype(np.int32))
        col = pinned_copy(torch, np.ascontiguousarray(g.col, dtype=np.int32))
        pinned.append((g.n, rp.numpy(), col.numpy(), rp, col))
    with T.Context(dev.index) as c:  # every graph counted alone first
        alone = [c.count(n, rp.to(dev), col.to(dev)) for n, _, _, rp, col in pinned]
    rng = np.random.default_rng(SERVE["seed"])
    n_req = max(1, int(SERVE["rate"] * seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / SERVE["rate"], n_req))
    pick = np.where(rng.random(n_req) < SERVE["big_fraction"], len(pool) + rng.integers(0, len(big), n_req),
                    rng.integers(0, len(pool), n_req))
    edges = sum(graphs[i].m for i in pick)

    def trace_loop(submit, poll):
        """Submit request i at arrivals[i]; collect completions as they come."""
        submit_t = np.zeros(n_req)
        done_t = np.zeros(n_req)
        result = [None] * n_req
        outstanding = {}
        nxt = 0
        t0 = time.perf_counter()
        while nxt < n_req or outstanding:
            now = time.perf_counter() - t0
            while nxt < n_req and arrivals[nxt] <= now:
                outstanding[submit(pick[nxt])] = nxt
                submit_t[nxt] = time.perf_counter() - t0
                nxt += 1
            for tk in list(outstanding):
                v = poll(tk)
                if v is not None:
                    i = outstanding.pop(tk)
                    done_t[i] = time.perf_counter() - t0
                    result[i] = v
            if nxt < n_req and not outstanding:
                time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.001)))
        return submit_t, done_t, result

    with T.Context(dev.index, mem_budget=SERVE["budget_gb"] << 30) as c:
        warm = c.submit_borrowed(pinned[0][0], pinned[0][1], pinned[0][2])  # starts the serving worker
        c.drain()
        assert c.poll(warm) == alone[0]
        submit_t, done_t, result = trace_loop(lambda j: c.submit_borrowed(*pinned[j][:3]), c.poll)
    lat = (done_t - submit_t) * 1e3
    span = done_t.max() - submit_t.min()
    served = {"graphs_per_s": n_req / span, "edges_per_s": edges / span, "span_s": span, **_percentiles(lat)}

    # capacity: the first `sat` requests of the trace submitted back to back
    sat = min(n_req, 20000)
    with T.Context(dev.index, mem_budget=SERVE["budget_gb"] << 30) as c:
        warm = c.submit_borrowed(*pinned[0][:3])
        c.drain()
        c.poll(warm)
        t = time.perf_counter()
        tickets = [c.submit_borrowed(*pinned[pick[i]][:3]) for i in range(sat)]
        c.drain()
        sat_s = time.perf_counter() - t
        sat_ok = all(c.poll(tk) == alone[pick[i]] for i, tk in enumerate(tickets))

    # the plain per-graph call on the same trace: tc_count_host, one at a time
    with T.Context(dev.index) as c:
        for j in range(len(pool), len(graphs)):  # grow the workspace for the largest graphs
            c.count_host(*pinned[j][:3])
        t = time.perf_counter()
        sat_loop_ok = all(c.count_host(*pinned[pick[i]][:3]) == alone[pick[i]] for i in range(sat))
        sat_loop_s = time.perf_counter() - t
        done = {}

        def submit_loop(j):
            k = len(done)
            done[k] = c.count_host(*pinned[j][:3])
            return k

        l_submit, l_done, l_result = trace_loop(submit_loop, lambda k: done.pop(k))
    # a request of the loop waits for the ones before it: its latency runs from its arrival
    l_lat = (l_done - arrivals) * 1e3
    l_span = l_done.max() - arrivals.min()
    return {
        "arrival_rate_per_s": SERVE["rate"], "seconds": seconds, "requests": n_req,
        "big_requests": int((pick >= len(pool)).sum()), "budget_gb": SERVE["budget_gb"],
        "draws": f"{len(pool)} independent draws of the batched distribution (uniform) + "
                 f"{len(big)} R-MAT scale-{SERVE['big_scale']} graphs",
        **served, "delivered_fraction": (n_req / span) / SERVE["rate"],
        "identical_to_alone": all(result[i] == alone[pick[i]] for i in range(n_req)),
        "submission": "tc_submit_borrowed from pinned host memory",
        "loop": {"api": "tc_count_host per request, in arrival order", "graphs_per_s": n_req / l_span,
                 "span_s": l_span, **_percentiles(l_lat),
                 "identical_to_alone": all(l_result[i] == alone[pick[i]] for i in range(n_req))},
        "served_vs_loop_graphs_per_s": (n_req / span) / (n_req / l_span),
        "saturation": {"requests": sat, "note": "the trace's first requests submitted back to back",
                       "served_graphs_per_s": sat / sat_s, "loop_graphs_per_s": sat / sat_loop_s,
                       "served_vs_loop": sat_loop_s / sat_s, "identical_to_alone": sat_ok and sat_loop_ok},
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

def pinned_copy(torch, a):
    """A page-locked host copy of numpy array `a` (allocated page-locked,
    then filled)."""
    t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
    t.copy_(torch.from_numpy(a))
    return t


class HugePinned:
    """A page-locked host copy of a large numpy array in 2 MiB pages: anonymous
    memory mapped with madvise(MADV_HUGEPAGE), filled, then registered with
    cudaHostRegister. On the GB300 machine the copy engine read such buffers at
    209-211 GB/s when (nearly) all of them sat in 2 MiB pages, and at 18-65
    GB/s when 4-11 % of them had fallen back to 4 KiB pages, which happens when
    they are first touched after the graph generation has churned host memory;
    HugePinned.reserve() maps and touches a region before that, and the
    constructor fills a reserved region when one large enough is given.
    `array` is the host view; close() unregisters and unmaps."""

    _libc = None

    @classmethod
    def _c(cls):
        import ctypes
        if cls._libc is None:
            libc = ctypes.CDLL("libc.so.6", use_errno=True)
            libc.mmap.restype = ctypes.c_void_p
            libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_long]
            libc.madvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
            libc.memset.restype = ctypes.c_void_p
            libc.memset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t]
            cls._libc = libc
        return cls._libc

    @classmethod
    def reserve(cls, nbytes: int):
        """Map `nbytes` (rounded up to 2 MiB) of anonymous memory, advise huge
        pages and touch every page now. Returns (ptr, nbytes)."""
        import ctypes
        libc = cls._c()
        nbytes = max((int(nbytes) + (2 << 20) - 1) // (2 << 20) * (2 << 20), 2 << 20)
        p = libc.mmap(None, nbytes, 3, 0x22, -1, 0)  # PROT_READ|PROT_WRITE, MAP_PRIVATE|MAP_ANONYMOUS
        if p in (None, ctypes.c_void_p(-1).value):
            raise MemoryError("mmap failed")
        libc.madvise(p, nbytes, 14)  # MADV_HUGEPAGE (advice only; 4 KiB pages still work)
        libc.memset(p, 0, nbytes)
        return p, nbytes

    def __init__(self, torch, a, region=None):
        import ctypes

        import numpy as np
        self._cudart = torch.cuda.cudart()
        if region is not None and region[1] >= a.nbytes:
            self.ptr, self.nbytes = region
        else:
            if region is not None:
                self._c().munmap(region[0], region[1])
            self.ptr, self.nbytes = self.reserve(a.nbytes)
        p = self.ptr
        buf = (ctypes.c_char * self.nbytes).from_address(p)
        self.array = np.frombuffer(buf, dtype=a.dtype, count=a.size)
        self.array[:] = a.reshape(-1)
        err = self._cudart.cudaHostRegister(p, self.nbytes, 0)
        self.registered = int(err) == 0 if not hasattr(err, "value") else err.value == 0
        if not self.registered:
            raise RuntimeError(f"cudaHostRegister failed: {err}")

    def hugepage_fraction(self) -> float:
        """Share of the buffer in transparent huge pages (/proc/self/smaps)."""
        import re
        huge, cur = 0, False
        try:
            for line in open("/proc/self/smaps"):
                m = re.match(r"([0-9a-f]+)-([0-9a-f]+) ", line)
                if m:
                    a, b = int(m.group(1), 16), int(m.group(2), 16)
                    cur = a < self.ptr + self.nbytes and self.ptr < b
                elif cur and line.startswith("AnonHugePages:"):
                    huge += int(line.split()[1]) * 1024
        except OSError:
            return -1.0
        return huge / self.nbytes

    def close(self):
        if self.ptr:
            if self.registered:
                self._cudart.cudaHostUnregister(self.ptr)
            self.array = None
            self._c().munmap(self.ptr, self.nbytes)
            self.ptr = None


def measure_graph(T, torch, dev, key, spec, g, steps, warmup, rank, world, dist, e2e_steps, clocks,
                  regions=(None, None)):
    """Time `steps` device steps (tc_count_async) of graph g after `warmup`
    untimed ones, then the end-to-end call (tc_count_host from pinned host
    memory, copies inside the timed region). Returns the line's keys, the
    context-side statistics and the counts."""
    import numpy as np

    from paper_2103_08053_gb300 import shard
    bits = spec["offset_bits"]
    if bits == 32 and g.nnz >= 2 ** 31:
        bits = 64
    rp_h = g.row_ptr.astype(np.int32 if bits == 32 else np.int64)
    col_h = np.ascontiguousarray(g.col, dtype=np.int32)
    rp = torch.from_numpy(rp_h).to(dev)
    col = torch.from_numpy(col_h).to(dev)
    ctx = T.Context(dev.index, params=dict(record_timing=1, **shard.shard_params(rank, world)))
    stream = torch.cuda.current_stream(dev)

    # exact statistics of the DAG (outside the timed region): W+ for the byte model
    with T.Context(dev.index) as full:
        dag = full.orient(g.n, rp, col)
        st = full.dag_stats(dag)
        dag.free()

    out = torch.zeros(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(warmup):
        ctx.count_async(g.n, rp, col, out, err, stream=stream)
    torch.cuda.synchronize(dev)
    my_count = int(out.item())
    if int(err.item()) != 0:
        raise SystemExit(f"counting failed with status {int(err.item())}")
    ctx.read_timing()  # drop warm-up timings
    launches0 = ctx.kernel_launches()

    sampler = ClockSampler(dev.index) if clocks else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.count_async(g.n, rp, col, out, err, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = sampler.stop() if sampler else None
    elapsed_ms = e0.elapsed_time(e1)
    launches = ctx.kernel_launches() - launches0
    tm = ctx.read_timing()
    total_count, elapsed_ms = shard.combine(my_count, elapsed_ms, device=dev)
    ms_per_step = elapsed_ms / steps

    # end to end through the C ABI from pinned host memory: H2D of the CSR, the
    # whole path, D2H of the count, every step
    rp_hp, col_hp = HugePinned(torch, rp_h, regions[0]), HugePinned(torch, col_h, regions[1])
    rp_pin, col_pin = torch.from_numpy(rp_hp.array), torch.from_numpy(col_hp.array)
    for _ in range(3):
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
    huge = col_hp.hugepage_fraction()
    del rp_d, col_d, rp_pin, col_pin
    rp_hp.close()
    col_hp.close()
    ctx.read_timing()
    ctx.close()

    peak, peak_src = measured_hbm_peak()
    calls = max(tm["calls"], 1)
    count_ms = tm["count_ms"] / calls
    bytes_count = count_phase_bytes(g.n, g.m, st["wedges_plus"])
    achieved = bytes_count / (count_ms / 1e3) / 1e9
    line = {
        "value": g.m / (ms_per_step / 1e3), "ms_per_step": ms_per_step,
        "config": {
            "workload": spec["name"], "n": g.n, "m": g.m, "nnz": g.nnz, "offset_bits": bits,
            "triangles": total_count, "wedges_plus": st["wedges_plus"], "max_out_degree": st["max_out_degree"],
            "bins": {"skip": st["n_skip"], "warp": st["n_warp"], "block": st["n_block"],
                     "wedges_plus_block": st["wedges_plus_block"]},
            "step": "tc_count_async: orientation + binning + hash build/probe + reduction, CSR resident in HBM",
            "l2": "no flush: inputs larger than L2 (col %.2f GB, DAG %.2f GB vs 129 MB)"
                  % (g.nnz * 4 / 1e9, (g.m + g.n) * 4 / 1e9),
            "parallelism": f"workload partition u % {world}" if world > 1 else "single GPU",
        },
        "phases_ms": {"orient": tm["orient_ms"] / calls, "bin": tm["bin_ms"] / calls, "count": count_ms},
        "roofline": {"kernel": "counting kernels (k_count_block + k_count_pack)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                     else "fallback 6.8 TB/s", "traffic": profiled_traffic(key),
                     "algorithmic_bytes_per_launch": bytes_count,
                     "bytes_model": "4(n+1) + 12m + 4W+ per counting step"},
        "e2e": {"value": g.m / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "stat": f"median of {e2e_steps} timed calls", "mean_ms_per_step": e2e_mean_ms,
                "max_ms_per_step": max(e2e_each),
                "h2d_bytes_per_step": int(rp_h.nbytes + col_h.nbytes), "d2h_bytes_per_step": 16,
                "h2d_copy_ms": h2d_ms, "host_pinned": "cudaHostRegister of 2 MiB-page (madvise) host buffers",
                "host_hugepage_fraction": round(huge, 3),
                "count_equal_device": e2e_count == my_count,
                "api": "tc_count_host (pinned host CSR)"},
        "gpu_launches": launches,
    }
    if clk is not None:
        line["clocks"] = clk
    return line, (rp, col), total_count


def bernoulli_sample(n: int, fraction: float, seed: int):
    """Vertex ids, each kept independently with probability `fraction`. (An
    arithmetic progression of ids would not do: R-MAT degrees depend on the
    bits of an id, so ids equal modulo a power of two share a degree class.)"""
    import numpy as np
    return np.flatnonzero(np.random.default_rng(seed).random(n) < fraction).astype(np.int64)


def oracle_baseline(g, fraction: float, seed: int = 7):
    """The CPU oracle on the host cores: orientation of the whole graph, then
    apex counts of every vertex (fraction 1) or of a Bernoulli sample of
    `fraction` of the vertices, whose time divided by `fraction` estimates
    the whole graph's. Returns (cpu_baseline, sampled vertices, their apex
    counts, total or None)."""
    import numpy as np

    import oracle
    cores = oracle.max_threads()
    t = time.perf_counter()
    d = oracle.orient(g)
    t_orient = time.perf_counter() - t
    if fraction >= 1.0:
        t = time.perf_counter()
        total, pv = oracle.count_dag(d, per_vertex=True, threads=cores)
        t_count = time.perf_counter() - t
        us, apex = np.arange(g.n), pv
        est = t_orient + t_count
        sample = (f"one oracle orientation + node-iterator count of the whole {g.name or 'graph'} "
                  f"({est:.1f} s)")
    else:
        us = bernoulli_sample(g.n, fraction, seed)
        t = time.perf_counter()
        apex = oracle.count_dag_at(d, us, threads=cores)
        t_count = time.perf_counter() - t
        total = None
        est = t_orient + t_count / fraction
        sample = (f"oracle orientation of the whole graph ({t_orient:.1f} s) + apex counts of a Bernoulli "
                  f"sample of the vertices with probability {fraction:g} ({len(us)} vertices, {t_count:.1f} s), "
                  f"the count time divided by {fraction:g}: {est:.1f} s for the whole graph")
    cb = {"value": g.m / est, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
          "seconds_whole_graph": est}
    return cb, us, apex, total


def run_gb300(args):
    import numpy as np
    import torch

    import graphgen as G
    import paper_2103_08053_gb300 as T

    rank, local_rank, world = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    key = args.workload
    spec = WORKLOADS[key]
    single = world == 1

    # host buffers of the end-to-end calls, mapped and touched before the
    # graph generation churns host memory, so that they get 2 MiB pages
    regions = host_regions(spec)
    regions2 = host_regions(WORKLOADS["rgg22"]) if single and args.second and key != "rgg22" else (None, None)
    t0 = time.time()
    g = make_graph(spec)
    g.name = spec["name"]
    log(f"[rank {rank}] generated {spec['name']}: n={g.n} m={g.m} in {time.time() - t0:.1f}s")
    main, (rp, col), total = measure_graph(T, torch, dev, key, spec, g, args.steps, args.warmup, rank, world,
                                           dist, e2e_steps=max(3, min(args.steps, args.e2e_steps)), clocks=True,
                                           regions=regions)
    log(f"[rank {rank}] {spec['name']}: {main['ms_per_step']:.2f} ms per step")
    result = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        **{k: main[k] for k in ("config", "phases_ms", "roofline", "e2e", "gpu_launches", "clocks")},
    }
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # the CPU baseline, the parity checks, the second workload, the batched,
    # served and study sections are single-GPU measurements: a multi-rank run
    # reports the sharded step only
    if single:
        parity = {"gpu": total}
        if spec.get("golden"):
            want = json.load(open(os.path.join(GOLDEN, spec["golden"])))
            parity.update({"golden": f"tests/golden/{spec['golden']}", "oracle": want["triangles"],
                           "equal": want["triangles"] == total,
                           "wedges_plus_equal": want["wedges_plus"] == main["config"]["wedges_plus"]})
        if not args.no_cpu_baseline:
            cb, us, apex, want_total = oracle_baseline(g, spec["oracle_fraction"])
            result["cpu_baseline"] = cb
            # the GPU's per-vertex apex counts at the oracle's sampled vertices
            with T.Context(dev.index) as c:
                d = c.orient(g.n, rp, col)
                pv = torch.zeros(g.n, dtype=torch.int64, device=dev)
                c.count_dag(d, per_vertex=pv)
                d.free()
            got = pv[torch.from_numpy(us).to(dev)].cpu().numpy().view(np.uint64)
            del pv
            parity["oracle_apex_vertices"] = int(len(us))
            parity["oracle_apex_equal"] = bool(np.array_equal(got, apex))
            if want_total is not None:
                parity.update({"oracle": want_total, "equal": want_total == total})
        result["parity"] = parity
    del rp, col
    torch.cuda.empty_cache()

    if single and args.second and key != "rgg22":
        s2 = WORKLOADS["rgg22"]
        g2 = make_graph(s2)
        g2.name = s2["name"]
        line2, (rp2, col2), total2 = measure_graph(T, torch, dev, "rgg22", s2, g2, 50, 5, 0, 1, None, e2e_steps=10,
                                                   clocks=False, regions=regions2)
        import oracle
        t = time.perf_counter()
        want2 = oracle.count(g2, threads=oracle.max_threads())
        cpu2 = time.perf_counter() - t
        line2["cpu_baseline"] = {"value": g2.m / cpu2, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                                 "sample": f"one oracle orientation + node-iterator count of the whole graph "
                                           f"({cpu2:.1f} s)"}
        line2["parity"] = {"oracle": want2, "gpu": total2, "equal": want2 == total2}
        result["rgg22"] = line2
        studies_rgg = (g2, rp2, col2)
    elif single and key == "rgg22":
        studies_rgg = (g, *make_graph_tensors(torch, dev, g))
    else:
        studies_rgg = None

    pool = None
    if single and (args.batched or args.serve_seconds > 0):
        t = time.time()
        pool = G.batch(BATCH["seed"], BATCH["graphs"])
        log(f"generated {BATCH['name']} in {time.time() - t:.1f}s")
    if args.batched and single:
        result["batched"] = measure_batched(T, torch, dev, args.batch_steps, pool)
        result["batched"]["generation_s"] = round(time.time() - t, 1)
    if args.serve_seconds > 0 and single:
        result["serving"] = measure_serving(T, torch, dev, args.serve_seconds, pool)
    del pool
    if args.reorder and single and studies_rgg:
        big = G.rmat(22, 16, seed=5)
        gs = {WORKLOADS["rgg22"]["name"]: (studies_rgg[0].n, studies_rgg[1], studies_rgg[2]),
              "rmat-s22-ef16-seed5": (big.n, *make_graph_tensors(torch, dev, big))}
        result["reorder_study"] = measure_reorder(T, torch, dev, gs)
    if args.ablation and single and studies_rgg:
        small = G.workload("rmat16")
        gs = {WORKLOADS["rgg22"]["name"]: (studies_rgg[0].n, studies_rgg[1], studies_rgg[2]),
              WORKLOADS["rmat16"]["name"]: (small.n, *make_graph_tensors(torch, dev, small))}
        result["ablation_study"] = measure_ablation(T, torch, dev, gs)
    if dist:
        dist.destroy_process_group()
    print(json.dumps(result), flush=True)


def host_regions(spec):
    """HugePinned reservations for a workload's row offsets and neighbour
    lists, sized by the workload's bounds on n and nnz."""
    bits = spec["offset_bits"]
    return (HugePinned.reserve((spec["n"] + 1) * bits // 8), HugePinned.reserve(spec["nnz_max"] * 4))


def make_graph_tensors(torch, dev, g):
    import numpy as np
    return (torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(dev))


def run_reference(args):
    """The oracle as it stands, on the host cores, on the main workload: the
    whole graph is oriented once (timed), then every step counts the apex
    triangles of a fresh systematic sample of REF_FRACTION of the vertices;
    a step's value is the whole-graph TEPS it implies (orientation time +
    sample time / REF_FRACTION)."""
    rank, _, world = dist_env()
    if rank != 0:
        return  # the CPU oracle runs once, on rank 0
    import numpy as np

    import oracle
    spec = WORKLOADS[args.workload]
    g = make_graph(spec)
    # rank 0 alone does the work: all host cores, whatever OMP_NUM_THREADS
    # the launcher set for its ranks
    cores = max(oracle.max_threads(), len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                else (os.cpu_count() or 1))
    t = time.perf_counter()
    d = oracle.orient(g)
    t_orient = time.perf_counter() - t
    frac = REF_FRACTION if spec["oracle_fraction"] < 1 else 1.0
    seeds = iter(range(11, 11 + args.warmup + args.steps))

    def step():
        us = bernoulli_sample(g.n, frac, next(seeds)) if frac < 1 else np.arange(g.n, dtype=np.int64)
        t = time.perf_counter()
        oracle.count_dag_at(d, us, threads=cores)
        return time.perf_counter() - t

    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    value = g.m / (t_orient + ms / 1e3 / frac)
    sample = (f"oracle orientation of the whole {spec['name']} graph once ({t_orient:.1f} s), then per step the "
              f"apex counts of a fresh Bernoulli sample of the vertices with probability {frac:g}, {cores} threads; "
              f"value = m / (orientation + step time / {frac:g})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": spec["name"], "n": g.n, "m": g.m, "sample_fraction": frac,
                   "orientation_s": t_orient},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=list(WORKLOADS), default=DEFAULT_WORKLOAD,
                    help="graph of the timed steps (default: R-MAT scale 26 with int64 row offsets); the second "
                         "workload, batched, serving and study sections use their own graphs")
    ap.add_argument("--e2e-steps", type=int, default=5, help="timed end-to-end calls (at most --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--second", type=int, default=1,
                    help="1: also time the RGG 2^22 workload (rank 0) when it is not the main one")
    ap.add_argument("--batched", type=int, default=1, help="1: also time the 4096-graph batch (rank 0)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--ablation", type=int, default=1,
                    help="1: also run the Sec. 3.3 (build/probe, edge-centric) and Sec. 4.2 (WC/SW/PC/VC) ablations (rank 0)")
    ap.add_argument("--reorder", type=int, default=1,
                    help="1: also run the Sec. 4.1 reordering study (rank 0)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="seconds of Poisson arrivals for the serving measurement (0: skip)")
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
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
