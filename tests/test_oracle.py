"""Pins of the CPU oracle against facts that do not come from the oracle.

Every check here compares the oracle with something independent of it: the
definition (brute force), linear algebra (trace(A^3)/6), closed forms of
graph families, invariances of the count, the paper's own worked examples
(tests/golden), and a statistical expectation. A dropped term, a wrong
comparison, a non-strict order or a transposed operand in the oracle fails at
least one of them.
"""
import itertools
import json
import math
from fractions import Fraction
import os

import numpy as np
import pytest

import graphgen as G
import oracle
from oracle import alg1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _graph_from_mask(n, mask):
    pairs = list(itertools.combinations(range(n), 2))
    e = [pairs[k] for k in range(len(pairs)) if (mask >> k) & 1]
    return G.from_edge_list(n, e) if e else G.empty(n)


# ---------------------------------------------------------------- definition

def test_brute_force_closed_forms():
    # the brute force itself is pinned by C(n,3) on K_n and 0 on K_{a,b}
    for n in range(0, 12):
        assert oracle.brute(G.complete(n) if n > 1 else G.empty(n)) == math.comb(n, 3)
    assert oracle.brute(G.complete_bipartite(5, 7)) == 0


@pytest.mark.parametrize("n", [3, 4, 5])
def test_exhaustive_small_graphs(n):
    # every labelled graph on n vertices: oracle == definition
    for mask in range(1 << (n * (n - 1) // 2)):
        g = _graph_from_mask(n, mask)
        assert oracle.count(g) == oracle.brute(g), (n, mask)


def test_random_subset_n7():
    rng = np.random.default_rng(7)
    for mask in rng.integers(0, 1 << 21, size=600):
        g = _graph_from_mask(7, int(mask))
        assert oracle.count(g) == oracle.brute(g), int(mask)


@pytest.mark.parametrize("n,p,seed", [(30, 0.3, 1), (60, 0.5, 2), (120, 0.1, 3), (200, 0.05, 4), (200, 0.6, 5)])
def test_random_gnp_vs_brute(n, p, seed):
    g = G.random_small(n, p, seed)
    assert oracle.count(g) == oracle.brute(g)


# ----------------------------------------------------------------- algebra

@pytest.mark.parametrize("n,p,seed", [(50, 0.2, 11), (256, 0.08, 12), (512, 0.03, 13), (300, 0.5, 14)])
def test_trace_a_cubed(n, p, seed):
    g = G.random_small(n, p, seed)
    a = np.zeros((n, n), dtype=np.int64)
    src = np.repeat(np.arange(n), np.diff(g.row_ptr))
    a[src, g.col] = 1
    tr = int(np.trace(a @ a @ a))
    assert tr % 6 == 0
    assert oracle.count(g) == tr // 6


# ------------------------------------------------------------ closed forms

def test_closed_forms():
    for n in range(3, 41):
        assert oracle.count(G.complete(n)) == math.comb(n, 3)
    assert oracle.count(G.cycle(3)) == 1
    for n in range(4, 30):
        assert oracle.count(G.cycle(n)) == 0
    for n in range(4, 30):
        assert oracle.count(G.wheel(n)) == n            # hub + every rim edge
    assert oracle.count(G.wheel(3)) == 4                # W_3 = K_4
    for k in range(1, 20):
        assert oracle.count(G.friendship(k)) == k
    for a, b in [(1, 1), (3, 4), (10, 10), (1, 50)]:
        assert oracle.count(G.complete_bipartite(a, b)) == 0
    for a, b in [(2, 2), (5, 7), (30, 30)]:
        assert oracle.count(G.grid2d(a, b)) == 0
    for s in (4, 5, 8, 16):
        assert oracle.count(G.torus3d(s)) == 0
    assert oracle.count(G.torus3d(3)) == 27             # every axis ring of a 3^3 torus is a triangle
    assert oracle.count(G.star(100)) == 0
    assert oracle.count(G.empty(10)) == 0


def test_3d_torus_scaled_like_dataset_row():
    # The dataset table's 3Dgrid row is a 464^3 periodic grid with |E| = 3|V|
    # and no triangles; the same family at a size the CPU suite can afford.
    row = json.load(open(os.path.join(GOLDEN, "dataset_3dgrid.json")))
    assert 464 ** 3 == row["V"] and 3 * 464 ** 3 == row["E"]
    g = G.torus3d(64)
    assert g.m == 3 * g.n
    assert oracle.count(g) == row["triangles"]


# --------------------------------------------------------------- invariance

@pytest.mark.parametrize("seed", [21, 22, 23])
def test_relabel_invariance(seed):
    g = G.rmat(10, 8, seed=seed)
    t = oracle.count(g)
    perm = np.random.default_rng(seed).permutation(g.n)
    assert oracle.count(G.relabel(g, perm)) == t
    assert t > 0


def test_row_order_invariance():
    g = G.rmat(10, 8, seed=31)
    assert oracle.count(G.shuffle_rows(g, 5)) == oracle.count(g)


@pytest.mark.parametrize("which", ["id", "reverse_id", "random"])
def test_orientation_order_invariance(which):
    g = G.rmat(9, 12, seed=41)
    n = g.n
    key = {"id": np.arange(n), "reverse_id": n - np.arange(n),
           "random": np.random.default_rng(3).permutation(n)}[which]
    d = oracle.orient(g, key=key)
    assert oracle.count_dag(d) == oracle.count(g) == oracle.brute(g)


def test_disjoint_union_additivity():
    gs = [G.rmat(8, 8, seed=s) for s in range(5)] + [G.complete(9), G.wheel(12), G.empty(3)]
    assert oracle.count(G.disjoint_union(gs)) == sum(oracle.count(g) for g in gs)


# --------------------------------------------------------------- orientation

def test_orientation_keeps_each_edge_once_towards_higher_rank():
    g = G.rmat(11, 8, seed=51)
    d = oracle.orient(g)
    deg = g.degrees()
    assert d.m == g.m
    src = np.repeat(np.arange(g.n), d.out_degrees())
    dst = d.dag_col.astype(np.int64)
    rank_lt = (deg[src] < deg[dst]) | ((deg[src] == deg[dst]) & (src < dst))
    assert rank_lt.all()
    und = set(zip(np.minimum(src, dst).tolist(), np.maximum(src, dst).tolist()))
    assert len(und) == g.m
    # rows sorted
    for u in range(0, g.n, 97):
        r = d.dag_col[d.dag_ptr[u]:d.dag_ptr[u + 1]]
        assert (np.diff(r) > 0).all()
    # out-degree bound from the degree order: d+(u)^2 <= 2|E|
    assert int(d.out_degrees().max()) ** 2 <= 2 * g.m


def test_per_vertex_counts():
    g = G.random_small(40, 0.3, 61)
    d = oracle.orient(g)
    t, pv = oracle.count_dag(d, per_vertex=True)
    assert int(pv.sum()) == t == oracle.brute(g)
    # apex(u) by brute force: triangles whose lowest vertex in the order is u
    deg = g.degrees()
    rank = {u: (int(deg[u]), u) for u in range(g.n)}
    adj = {u: set(g.row(u).tolist()) for u in range(g.n)}
    want = np.zeros(g.n, dtype=np.uint64)
    for a, b, c in itertools.combinations(range(g.n), 3):
        if b in adj[a] and c in adj[b] and c in adj[a]:
            want[min((a, b, c), key=lambda x: rank[x])] += 1
    assert (pv == want).all()
    us = np.array([0, 5, 17, 39])
    assert (oracle.count_dag_at(d, us) == want[us]).all()


def test_threaded_equals_single_thread():
    g = G.rmat(12, 16, seed=71)
    assert oracle.count(g, threads=1) == oracle.count(g, threads=0)


# ------------------------------------------------------- Algorithm 1 reading

@pytest.mark.parametrize("B,L", [(32, 128), (4, 8), (1, 64), (16, 2), (64, 3), (2, 16)])
def test_alg1_reading_equals_oracle(B, L):
    g = G.rmat(8, 8, seed=81)
    d = oracle.orient(g)
    if B * L <= int(d.out_degrees().max()):
        pytest.skip("table smaller than the largest out-list")
    assert alg1.count_alg1(d.dag_ptr.tolist(), d.dag_col.tolist(), B, L) == oracle.count(g)


def test_alg1_overflow_chain():
    # every key lands in bucket 0; with L = 2 the keys chain through buckets 1, 2, ...
    t = alg1.hash_table_construction([0, 16, 32, 48, 64, 80, 96], B=16, L=2)
    assert t.length[:4] == [2, 2, 2, 1] and t.length[4:] == [0] * 12
    for k in [0, 16, 32, 48, 64, 80, 96]:
        assert t.linear_search(k) == 1
    for k in [1, 112, 128, 5, 17]:
        assert t.linear_search(k) == 0


def test_vc_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "vc_example.json")))
    pre = alg1.inclusive_prefix(ex["degrees"])
    assert pre == ex["inclusive_prefix"]
    j, off = alg1.vc_locate(pre, ex["flat_index"])
    assert ex["neighbors_of_u"][j] == ex["owner_vertex"]
    assert off == ex["offset_in_owner"]
    lo = pre[j - 1] if j else 0
    assert [lo, pre[j]] == ex["owner_range"]
    # every flat index maps into its owner's range
    for k in range(pre[-1]):
        j, off = alg1.vc_locate(pre, k)
        assert 0 <= off < ex["degrees"][j]


def test_layout_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "layout_example.json")))
    B = ex["B"]
    t = alg1.BucketTable(B, max(len(b) for b in ex["buckets"]))
    # place each element in its printed bucket, in printed order (pins the
    # interleaving only; see the fixture's note on the hash)
    for i, bucket in enumerate(ex["buckets"]):
        for v in bucket:
            slot = t.length[i]
            t.length[i] += 1
            t.level[slot][i] = v
    assert t.flat() == ex["level_major_image"]
    # with the paper's hash (x % B) every element except 10 lands where printed
    t2 = alg1.hash_table_construction([v for b in ex["buckets"] for v in b if v != 10], B, 5)
    img = t2.flat()
    want = [x if x != 10 else None for x in ex["level_major_image"]]
    assert img == want


def test_cost_models():
    g = G.rmat(8, 8, seed=91)
    d = oracle.orient(g)
    dp, dc = d.dag_ptr.tolist(), d.dag_col.tolist()
    # Eq. 1 <= Eq. 2 (max collision bounds every bucket length); with one
    # bucket per possible key (B > n) Eq. 1 is the number of probes that hit,
    # i.e. the triangle count, and Eq. 2 is the collective degree W+.
    assert alg1.cost_eq1(dp, dc, 32, 128) <= alg1.phi_eq2(dp, dc, 32, 128)
    wplus = sum(alg1.collective_degree(dp, dc, u) for u in range(g.n))
    assert g.n <= 512
    assert alg1.cost_eq1(dp, dc, 512, 1) == oracle.count(g)
    assert alg1.phi_eq2(dp, dc, 512, 1) == wplus


# -------------------------------------------------------------- statistics

def test_gnp_expected_value_smoke():
    n, p = 400, 0.05
    ts = [oracle.count(G.erdos_renyi(n, p, seed=1000 + s)) for s in range(8)]
    expect = math.comb(n, 3) * p ** 3
    assert abs(np.mean(ts) - expect) < 4 * 75 / math.sqrt(len(ts))


# -------------------------------------------------------------- reordering

def test_reorder_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "reorder_example.json")))
    g = G.from_edge_list(ex["n"], [tuple(e) for e in ex["edges"]])
    assert np.diff(g.row_ptr).tolist() == ex["degrees"]
    d = oracle.orient(g)
    rows = [d.dag_col[d.dag_ptr[u]:d.dag_ptr[u + 1]].tolist() for u in range(g.n)]
    assert rows == ex["oriented_out_lists"]
    assert oracle.reorder(g, oracle.REORDER_INDEGREE).tolist() == ex["new_id_indegree"]
    assert oracle.reorder(g, oracle.REORDER_COLLECTIVE).tolist() == ex["new_id_collective"]
    for kind in (1, 2):
        h = oracle.relabel(g, oracle.reorder(g, kind))
        assert oracle.count(h) == oracle.brute(h) == ex["triangles"]


@pytest.mark.parametrize("seed", range(4))
def test_reorder_is_a_permutation_and_keeps_the_count(seed):
    g = G.rmat(9, 6 + seed, seed=300 + seed)
    want = oracle.count(g)
    for kind in (oracle.REORDER_INDEGREE, oracle.REORDER_COLLECTIVE):
        nid = oracle.reorder(g, kind)
        assert sorted(nid.tolist()) == list(range(g.n))
        h = oracle.relabel(g, nid)
        assert oracle.count(h) == want
        # the relabelled CSR is the same graph as graphgen's relabel builds
        r = G.relabel(g, nid)
        for u in range(g.n):
            a = sorted(h.col[h.row_ptr[u]:h.row_ptr[u + 1]].tolist())
            b = sorted(r.col[r.row_ptr[u]:r.row_ptr[u + 1]].tolist())
            assert a == b


def test_reorder_indegree_properties():
    g = G.rmat(10, 8, seed=311)
    d = oracle.orient(g)
    indeg = np.bincount(d.dag_col, minlength=g.n)
    nid = oracle.reorder(g, oracle.REORDER_INDEGREE)
    by_new = np.empty(g.n, dtype=np.int64)
    by_new[nid] = np.arange(g.n)          # old id of each new id
    seq = indeg[by_new]
    assert np.all(seq[:-1] >= seq[1:])    # largest in-degree first
    ties = seq[:-1] == seq[1:]
    assert np.all(by_new[:-1][ties] < by_new[1:][ties])  # ties by old id


def test_reorder_collective_properties():
    g = G.rmat(10, 8, seed=312)
    d = oracle.orient(g)
    dp, dc = d.dag_ptr, d.dag_col
    dplus = np.diff(dp)
    coll = np.array([dplus[dc[dp[u]:dp[u + 1]]].sum() for u in range(g.n)])
    top = int(np.lexsort((np.arange(g.n), -coll))[0])   # heaviest u, smallest id among ties
    nid = oracle.reorder(g, oracle.REORDER_COLLECTIVE)
    first = sorted(dc[dp[top]:dp[top + 1]].tolist())
    # the heaviest vertex's out-neighbours receive the first ids, in id order
    assert [int(nid[v]) for v in first] == list(range(len(first)))
    # vertices in no out-list get the last ids, in id order
    orphans = np.setdiff1d(np.arange(g.n), dc)
    assert nid[orphans].tolist() == list(range(g.n - len(orphans), g.n))


def test_collision_stats_against_algorithm1_tables():
    # with levels >= d+ no bucket overflows, so Algorithm 1's tables hold the
    # unbounded bucket loads and Eq. 2 from them must agree
    g = G.rmat(9, 8, seed=93)
    d = oracle.orient(g)
    dp, dc = d.dag_ptr.tolist(), d.dag_col.tolist()
    L = int(d.out_degrees().max())
    mx, phi = oracle.collision_stats(d, "mod32")
    assert phi == alg1.phi_eq2(dp, dc, 32, L)
    assert mx == max(alg1.hash_table_construction(dc[dp[u]:dp[u + 1]], 32, L).max_collision()
                     for u in range(g.n) if dp[u + 1] > dp[u])
    # a multiplicative hash of 32 consecutive ids spreads them over all buckets
    # (three-distance theorem: no bucket gets more than 2)
    h = G.star(40)          # every leaf's out-list is {hub}; the hub's is empty
    k = G.complete(34)      # N+(0) = {1..33}: consecutive ids
    dk = oracle.orient(k)
    assert oracle.collision_stats(dk, "mod32")[0] == 2          # 1 and 33 share bucket 1
    assert oracle.collision_stats(dk, "mult32")[0] <= 2
    assert oracle.collision_stats(oracle.orient(h), "mod32") == (1, 0)


def knuth_multiplicative_bucket(x: int, B: int) -> int:
    """Multiplicative hashing as Knuth defines it (TAOCP vol. 3, Sec. 6.4):
    h(K) = floor(M * frac(K * A / w)) with word size w = 2^32, M = B buckets
    and A the integer nearest w times the golden-ratio conjugate, taken
    prime; computed with exact fractions."""
    A = 2654435761
    return int(B * (Fraction(x * A, 2 ** 32) % 1))


def test_knuth_multiplier():
    A = 2654435761
    golden = (math.sqrt(5) - 1) / 2
    assert abs(A - 2 ** 32 * golden) < 10
    assert A % 2 and all(A % p for p in range(3, math.isqrt(A) + 1, 2))  # prime


def test_collision_stats_mult32_against_algorithm1_tables():
    # the "mult32" statistics are those of Algorithm 1's 32-bucket tables built
    # with Knuth's multiplicative hash instead of x mod 32: the largest bucket
    # load of any N+(u) and Eq. 2's phi from the same tables (levels >= d+:
    # nothing overflows, so the loads are the unbounded ones)
    for g in (G.rmat(9, 8, seed=93), G.rgg(600, 12.0, seed=94), G.complete(70)):
        d = oracle.orient(g)
        dp, dc = d.dag_ptr.tolist(), d.dag_col.tolist()
        L = max(1, int(d.out_degrees().max()))
        mx, phi = oracle.collision_stats(d, "mult32")
        assert phi == alg1.phi_eq2(dp, dc, 32, L, knuth_multiplicative_bucket)
        assert mx == max(alg1.hash_table_construction(dc[dp[u]:dp[u + 1]], 32, L,
                                                      knuth_multiplicative_bucket).max_collision()
                         for u in range(g.n) if dp[u + 1] > dp[u])
        # and the mod32 statistics of the same graphs against the plain tables
        mx0, phi0 = oracle.collision_stats(d, "mod32")
        assert phi0 == alg1.phi_eq2(dp, dc, 32, L)
