#!/usr/bin/env python3
"""Writes tests/golden/rmat26.json: the oracle's whole-graph triangle count of
the R-MAT scale-26 workload (edge factor 16, (a,b,c,d) = (0.57, 0.19, 0.19,
0.05), seed 3; self-loops dropped, deduplicated, symmetrised).

Only the seeded input generator (graphgen) and the CPU oracle run here: the
graph is generated, oriented by (degree, id) (Sec. 2.2) and counted by the
node iterator with merge intersection, all on the host. Besides the total it
records W+ = sum_u sum_{v in N+(u)} d+(v) (the number of 2-hop keys the
vertex-centric method probes, the oriented collective degree of Eq. 2), the
largest out-degree, and a SHA-256 digest of the per-vertex apex counts
apex(u) = sum_{v in N+(u)} |N+(u) ∩ N+(v)| as little-endian uint64, so a GPU
run can be compared with the oracle vertex by vertex without storing 67 M
numbers.

  python tests/golden/make_rmat26.py [--threads T]

Needs about 30 GB of host memory; the count takes minutes on 8 cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen as G  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat26.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    threads = args.threads or oracle.max_threads()
    t = time.time()
    g = G.workload("rmat26")
    gen_s = time.time() - t
    print(f"generated n={g.n} m={g.m} nnz={g.nnz} in {gen_s:.0f} s", flush=True)
    t = time.time()
    d = oracle.orient(g)
    orient_s = time.time() - t
    dplus = d.out_degrees()
    wplus = int(dplus[d.dag_col].astype(np.int64).sum())
    print(f"oriented in {orient_s:.0f} s: W+ = {wplus}", flush=True)
    t = time.time()
    total, per_vertex = oracle.count_dag(d, per_vertex=True, threads=threads)
    count_s = time.time() - t
    assert int(per_vertex.sum(dtype=np.uint64)) == total
    digest = hashlib.sha256(per_vertex.astype("<u8").tobytes()).hexdigest()
    rec = {
        "workload": "rmat-s26-ef16-seed3",
        "recipe": "graphgen.workload('rmat26'): R-MAT scale 26, 16 * 2^26 generated edges, (a,b,c,d) = "
                  "(0.57, 0.19, 0.19, 0.05), seed 3; self-loops dropped, deduplicated, symmetrised",
        "source": "written by tests/golden/make_rmat26.py from the CPU oracle alone (orientation by "
                  "(degree, id), Sec. 2.2; node iterator with merge intersection)",
        "n": g.n, "m": g.m, "nnz": g.nnz,
        "triangles": total,
        "wedges_plus": wplus,
        "max_out_degree": int(dplus.max()),
        "apex_sha256_le_u64": digest,
        "oracle_seconds": {"generate": round(gen_s, 1), "orient": round(orient_s, 1), "count": round(count_s, 1)},
        "oracle_threads": threads,
        "host": f"{platform.machine()}, {os.cpu_count()} cores",
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=2)
        f.write("\n")
    print(json.dumps(rec, indent=2))


if __name__ == "__main__":
    main()
