"""Parity at the workloads' full sizes, in the launch configuration bench.py
uses (default parameters, one context).

* the bench workload (RGG, 2^22 points, mean degree 64): whole count vs oracle;
* R-MAT scale 16: whole count vs oracle;
* R-MAT scale 26 with int64 offsets: the total, W+ and every vertex's apex
  count (by digest) against the oracle's, stored in tests/golden/rmat26.json,
  plus the oriented offsets and a sample of apex counts against the oracle run
  here;
* the 4096-graph batched workload: every graph's count vs the oracle, and the
  per-graph loop;
* the dataset table's 3Dgrid row (a 464^3 periodic grid): |V|, |E| and the
  count (0) exactly as printed.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as G
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as ge
    ge._load_builder().build()
    import paper_2103_08053_gb300 as T
    return T


def dev(g, bits=32):
    d = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int64 if bits == 64 else np.int32)).to(d)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d)
    return g.n, rp, col


def test_bench_workload_whole_count(T):
    g = G.workload("rgg22")
    want = oracle.count(g)
    with T.Context(0) as c:
        n, rp, col = dev(g)
        assert c.count(n, rp, col) == want
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        c.count_async(n, rp, col, out, err)
        torch.cuda.synchronize()
        assert int(out.item()) == want and int(err.item()) == 0


def test_rmat16_whole_count(T):
    g = G.workload("rmat16")
    with T.Context(0) as c:
        assert c.count(*dev(g)) == oracle.count(g)


def test_rmat26_whole_graph_against_the_oracle_golden(T):
    # tests/golden/rmat26.json holds the oracle's whole-graph count, W+ and a
    # digest of every vertex's apex count, written by tests/golden/make_rmat26.py
    # (graph generator + CPU oracle only)
    want = json.load(open(os.path.join(GOLDEN, "rmat26.json")))
    g = G.workload("rmat26")
    assert (g.n, g.m, g.nnz) == (want["n"], want["m"], want["nnz"])
    assert g.nnz > 1_000_000_000
    with T.Context(0) as c:
        n, rp, col = dev(g, 64)  # int64 row offsets, as the configuration states
        total = c.count(n, rp, col)
        assert total == want["triangles"]
        d = c.orient(n, rp, col)
        st = c.dag_stats(d)
        assert st["wedges_plus"] == want["wedges_plus"] and st["max_out_degree"] == want["max_out_degree"]
        pv = torch.zeros(n, dtype=torch.int64, device="cuda")
        assert c.count_dag(d, per_vertex=pv) == total
        got = pv.cpu().numpy().view(np.uint64)
        assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == want["apex_sha256_le_u64"]
        od = oracle.orient(g)
        assert d.m == od.m == g.m
        dp, _ = d.tensors()
        assert np.array_equal(dp.cpu().numpy().astype(np.int64), od.dag_ptr)
        deg = od.out_degrees()
        rng = np.random.default_rng(26)
        # every vertex with the largest out-degrees, plus a random sample
        us = np.unique(np.concatenate([np.argsort(deg)[-200:], rng.integers(0, n, 2000)]))
        want = oracle.count_dag_at(od, us)
        got = pv[torch.from_numpy(us).cuda()].cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, want)
        d.free()


def test_batched_workload_4096(T):
    gs = G.batch(4, 4096)
    want = oracle.count_many(gs)
    with T.Context(0) as c:
        tensors = [dev(g) for g in gs]
        counts = c.count_batch(tensors)
        assert counts == want  # every graph of the batch against the oracle
        assert [c.count(*t) for t in tensors] == want


def test_3dgrid_dataset_row(T):
    row = json.load(open(os.path.join(GOLDEN, "dataset_3dgrid.json")))
    g = G.torus3d(464)
    assert g.n == row["V"] and g.m == row["E"]
    with T.Context(0) as c:
        assert c.count(*dev(g)) == row["triangles"] == oracle.count(g)
