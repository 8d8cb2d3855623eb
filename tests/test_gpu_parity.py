"""CUDA path vs the CPU oracle, through the C ABI (bit-exact: counts are integers).

Inputs come from graphgen (seeded). Sizes span several scan tiles (8192
rows), several 32-row orientation groups with a ragged tail, warp and block
workers, multi-item and multi-part block work, and table overflow.
"""
import math

import numpy as np
import pytest

import graphgen as G
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as ge
    ge._load_builder().build()
    import paper_2103_08053_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctx(T):
    c = T.Context(0)
    yield c
    c.close()


def dev(g, bits=32):
    d = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int64 if bits == 64 else np.int32)).to(d)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d)
    return rp, col


def gpu_count(ctx, g, bits=32):
    rp, col = dev(g, bits)
    return ctx.count(g.n, rp, col)


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("make,want", [
    (lambda: G.complete(3), 1), (lambda: G.complete(40), math.comb(40, 3)),
    (lambda: G.complete(200), math.comb(200, 3)),      # d+ up to 199 -> block worker
    (lambda: G.cycle(3), 1), (lambda: G.cycle(1000), 0), (lambda: G.wheel(500), 500),
    (lambda: G.friendship(300), 300), (lambda: G.complete_bipartite(40, 60), 0),
    (lambda: G.grid2d(70, 90), 0), (lambda: G.torus3d(20), 0), (lambda: G.torus3d(3), 27),
    (lambda: G.star(5000), 0), (lambda: G.empty(7), 0),
])
def test_closed_forms(ctx, make, want):
    g = make()
    assert gpu_count(ctx, g) == want
    assert gpu_count(ctx, g, 64) == want


def test_tiny_and_empty(ctx):
    assert gpu_count(ctx, G.empty(0)) == 0
    assert gpu_count(ctx, G.empty(1)) == 0
    g = G.from_edge_list(2, [(0, 1)])
    assert gpu_count(ctx, g) == 0


# ----------------------------------------------------------- random graphs

@pytest.mark.parametrize("n,p,seed", [(30, 0.3, 1), (150, 0.2, 2), (200, 0.6, 3), (333, 0.05, 4)])
def test_random_small_vs_brute(ctx, n, p, seed):
    g = G.random_small(n, p, seed)
    want = oracle.brute(g)
    assert oracle.count(g) == want
    assert gpu_count(ctx, g) == want


@pytest.mark.parametrize("scale,ef,seed", [(8, 8, 1), (10, 16, 2), (13, 16, 3), (14, 4, 4), (15, 32, 5)])
def test_rmat_vs_oracle(ctx, scale, ef, seed):
    g = G.rmat(scale, ef, seed=seed)
    want = oracle.count(g)
    assert gpu_count(ctx, g) == want
    assert gpu_count(ctx, g, 64) == want


@pytest.mark.parametrize("n,seed", [(25_001, 6), (70_000, 7)])
def test_rgg_ragged_vs_oracle(ctx, n, seed):
    g = G.rgg(n, 48.0, seed=seed)
    assert gpu_count(ctx, g) == oracle.count(g)


def test_er_vs_oracle(ctx):
    g = G.erdos_renyi(20_011, 0.003, seed=8)
    assert gpu_count(ctx, g) == oracle.count(g)


def test_unsorted_rows_and_relabel(ctx):
    g = G.rmat(12, 16, seed=9)
    want = oracle.count(g)
    assert gpu_count(ctx, G.shuffle_rows(g, 1)) == want
    perm = np.random.default_rng(2).permutation(g.n)
    assert gpu_count(ctx, G.relabel(g, perm)) == want


def test_disjoint_union(ctx):
    gs = [G.rmat(9, 8, seed=s) for s in range(4)] + [G.complete(150), G.wheel(64)]
    u = G.disjoint_union(gs)
    assert gpu_count(ctx, u) == sum(gpu_count(ctx, g) for g in gs) == oracle.count(u)


# --------------------------------------------------------------- the DAG

def test_orientation_matches_oracle(ctx):
    g = G.rmat(13, 16, seed=10)
    rp, col = dev(g)
    d = ctx.orient(g.n, rp, col)
    od = oracle.orient(g)
    assert d.m == od.m == g.m
    dp, dc = d.tensors()
    assert np.array_equal(dp.cpu().numpy().astype(np.int64), od.dag_ptr)
    # input rows are sorted and compaction keeps input order -> identical
    assert np.array_equal(dc.cpu().numpy(), od.dag_col)
    d.free()


def test_orientation_all_row_classes(ctx):
    # short rows (combined walk), rows of 129..1024 entries (one warp each) and
    # rows over 1024 (one block each), int32 and int64 offsets: the DAG must be
    # the oracle's entry for entry (input rows sorted, compaction keeps order)
    g = G.disjoint_union([G.star(3000), G.complete(400), G.rmat(12, 16, seed=31), G.star(700)])
    deg = np.diff(g.row_ptr)
    assert deg.max() > 1024 and ((deg > 128) & (deg <= 1024)).sum() > 100
    od = oracle.orient(g)
    for bits in (32, 64):
        rp, col = dev(g, bits)
        d = ctx.orient(g.n, rp, col)
        dp, dc = d.tensors()
        assert np.array_equal(dp.cpu().numpy().astype(np.int64), od.dag_ptr)
        assert np.array_equal(dc.cpu().numpy(), od.dag_col)
        d.free()
        assert gpu_count(ctx, g, bits) == oracle.count(g)


def test_orientation_unsorted_rows(ctx):
    g = G.shuffle_rows(G.rmat(11, 16, seed=11), 3)
    rp, col = dev(g)
    d = ctx.orient(g.n, rp, col)
    od = oracle.orient(g)
    dp, dc = d.tensors()
    dp, dc = dp.cpu().numpy(), dc.cpu().numpy()
    assert np.array_equal(dp.astype(np.int64), od.dag_ptr)
    for u in range(g.n):
        assert np.array_equal(np.sort(dc[dp[u]:dp[u + 1]]), od.dag_col[od.dag_ptr[u]:od.dag_ptr[u + 1]])
    d.free()


def test_per_vertex_counts(ctx):
    g = G.rmat(13, 16, seed=12)
    rp, col = dev(g)
    d = ctx.orient(g.n, rp, col)
    pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    total = ctx.count_dag(d, per_vertex=pv)
    want_total, want_pv = oracle.count_dag(oracle.orient(g), per_vertex=True)
    assert total == want_total
    assert np.array_equal(pv.cpu().numpy().astype(np.uint64), want_pv)
    st = ctx.dag_stats(d)
    od = oracle.orient(g)
    outd = od.out_degrees()
    assert st["m"] == od.m and st["max_out_degree"] == outd.max()
    assert st["wedges_plus"] == int(sum(outd[od.dag_col]))
    assert st["n_skip"] + st["n_warp"] + st["n_block"] == g.n
    d.free()


@pytest.mark.parametrize("balance", [1, 2, 3, 4])
def test_balance_modes_per_vertex_and_long_lists(T, balance):
    # per-vertex counts under each Sec. 4.2 alternative, on graphs whose 2-hop
    # lists are longer than a physical-combination round (stars joined to a
    # clique: a warp vertex whose out-neighbours have d+ in the thousands)
    hub = G.disjoint_union([G.complete(70), G.star(3000), G.rmat(12, 16, seed=21)])
    big = G.from_edge_list(2600, [(a, b) for a in range(2400, 2600) for b in range(a + 1, 2600)] +
                           [(a, b) for a in range(0, 2400) for b in range(2400, 2405)])
    for g in (hub, big):
        want_total, want_pv = oracle.count_dag(oracle.orient(g), per_vertex=True)
        with T.Context(0, params=dict(balance=balance)) as c:
            rp, col = dev(g)
            d = c.orient(g.n, rp, col)
            pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
            assert c.count_dag(d, per_vertex=pv) == want_total
            assert np.array_equal(pv.cpu().numpy().astype(np.uint64), want_pv)
            d.free()
            assert c.count(g.n, rp, col) == want_total
            assert c.count_batch([(g.n, rp, col), (g.n, rp, col)]) == [want_total, want_total]


@pytest.mark.parametrize("skewed", [True, False])
def test_octet_and_quad_builds_per_vertex(T, skewed):
    # both builds of the warp workers are launched and the graph's shape picks
    # one: with a small T_w most counted vertices become thread-block vertices
    # (the octet build works), with the default T_w the RGG graph has none (the
    # quad build works); per-vertex counts must equal the oracle's either way
    g = G.disjoint_union([G.rmat(13, 16, seed=44), G.rgg(20_000, 64.0, seed=45), G.complete(90)])
    want_total, want_pv = oracle.count_dag(oracle.orient(g), per_vertex=True)
    prm = dict(warp_max_out_degree=8, item_neighbors=32) if skewed else {}
    with T.Context(0, params=prm) as c:
        rp, col = dev(g)
        d = c.orient(g.n, rp, col)
        st = c.dag_stats(d)
        assert (100 * st["n_block"] >= st["n_warp"]) == skewed
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        assert c.count_dag(d, per_vertex=pv) == want_total
        assert np.array_equal(pv.cpu().numpy().astype(np.uint64), want_pv)
        d.free()
        assert c.count(g.n, rp, col) == want_total


def hub_spoke_graph(hubs=300, spokes=6000, per_spoke=8, seed=46):
    """A clique of `hubs` vertices and `spokes` small vertices, each joined to
    `per_spoke` random hubs. After orientation a spoke points at hubs (their
    degree is higher), whose out-lists within the clique average about
    hubs / 2 keys, and the hubs with d+ > 128 are thread-block vertices."""
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(hubs, 1)
    src = [i, np.repeat(np.arange(hubs, hubs + spokes), per_spoke)]
    dst = [j, np.concatenate([rng.choice(hubs, per_spoke, replace=False) for _ in range(spokes)])]
    return G.csr_from_edges(hubs + spokes, np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32))


def test_octet_path_of_the_warp_workers(T):
    # the warp workers' 32-byte octet loads run only in the octet build and only
    # for chunks whose 2-hop lists average at least 64 keys: here every spoke's
    # out-edges point at hubs with out-lists of about 150 keys, and about 170 of
    # the 6300 counted vertices are thread-block vertices (>= 1 %: the octet
    # build works); per-vertex counts against the oracle
    g = hub_spoke_graph()
    od = oracle.orient(g)
    spokes = np.arange(300, g.n)
    dplus = od.out_degrees()
    assert (dplus[spokes] == 8).all()
    lens = dplus[od.dag_col[od.dag_ptr[300]:]]
    assert lens.mean() >= 64
    want_total, want_pv = oracle.count_dag(od, per_vertex=True)
    with T.Context(0) as c:
        rp, col = dev(g)
        d = c.orient(g.n, rp, col)
        st = c.dag_stats(d)
        assert 100 * st["n_block"] >= st["n_warp"] and st["n_warp"] >= 6000
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        assert c.count_dag(d, per_vertex=pv) == want_total
        assert np.array_equal(pv.cpu().numpy().astype(np.uint64), want_pv)
        d.free()
        assert c.count(g.n, rp, col) == want_total


def test_unaligned_dag_and_ragged_quads(ctx):
    # wide loads need an aligned dag_col: 32-byte octets at shift 0, 16-byte
    # quads at shift 4 (16 bytes), one key per lane otherwise. All must equal
    # the oracle, including the per-vertex counts, and so must a DAG whose last
    # list ends at a length that is not a multiple of 4.
    g = G.rmat(12, 12, seed=21)
    od = oracle.orient(g)
    want_total, want_pv = oracle.count_dag(od, per_vertex=True)
    dp = torch.from_numpy(od.dag_ptr.astype(np.int32)).cuda()
    for shift in (0, 1, 2, 3, 4, 5):
        buf = torch.zeros(od.m + 8, dtype=torch.int32, device="cuda")
        buf[shift:shift + od.m] = torch.from_numpy(od.dag_col).cuda()
        dc = buf[shift:shift + od.m]
        raw = T_tc().tc_dag(g.n, od.m, dp.data_ptr(), dc.data_ptr())
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        assert ctx.count_dag(raw, per_vertex=pv) == want_total
        assert np.array_equal(pv.cpu().numpy().astype(np.uint64), want_pv)
    # a DAG cut right after a list whose end is not quad-aligned
    cut = next(u for u in range(g.n, 0, -1) if od.dag_ptr[u] % 4 != 0 and od.dag_ptr[u] > 0)
    sub_ptr = np.minimum(od.dag_ptr, od.dag_ptr[cut])
    sub = oracle.Dag(g.n, sub_ptr, od.dag_col[:od.dag_ptr[cut]].copy())
    exact = torch.from_numpy(sub.dag_col).cuda().clone()   # allocation of exactly m entries
    dps = torch.from_numpy(sub_ptr.astype(np.int32)).cuda()
    raw = T_tc().tc_dag(g.n, sub.m, dps.data_ptr(), exact.data_ptr())
    # keys in the truncated lists may name vertices >= cut whose lists are now empty
    assert ctx.count_dag(raw) == oracle.count_dag(sub)


def T_tc():
    from paper_2103_08053_gb300 import _tc
    return _tc


# ------------------------------------------------------ worker/table regimes

PARAM_SETS = {
    "tiny_block_items": dict(warp_max_out_degree=8, item_neighbors=32),  # many block items per vertex
    "one_table_per_pack": dict(warp_max_out_degree=12, warp_area_ints=144),
    "all_block": dict(warp_max_out_degree=1),                  # every vertex on the block path
    "all_warp": dict(warp_max_out_degree=255, warp_area_ints=2304, warps_per_block=4),
    "one_per_pop": dict(chunk=1),
    "big_min_buckets": dict(warp_min_buckets=512, warp_area_ints=2304),
    "small_items": dict(item_neighbors=32, warp_max_out_degree=16),
    "split_parts": dict(block_threads=64, block_smem_bytes=8192, item_neighbors=64, warp_max_out_degree=8),
    # ^ part_max = 256: out-lists longer than 256 are probed part by part
    "chunk7": dict(chunk=7, warp_area_ints=4608),
    "paper_hash": dict(hash_mode=1),
    "scalar_loads": dict(scalar_loads=1),                      # one 2-hop key per lane per load
    "edge_centric": dict(edge_centric=1),                      # Algorithm 2 ablation: a table per out-edge
    "cycle_timing": dict(record_timing=2),
    # Sec. 4.2's alternatives to virtual combination (warp workers)
    "balance_wc": dict(balance=1),
    "balance_sw8": dict(balance=2),
    "balance_sw16": dict(balance=3),
    "balance_pc": dict(balance=4),
    "balance_pc_small_packs": dict(balance=4, warp_max_out_degree=12, warp_area_ints=144, chunk=7),
    "balance_sw8_all_warp": dict(balance=2, warp_max_out_degree=255, warp_area_ints=2304, warps_per_block=4),
    # warp list grouped by the min-hash locality key (auto turns it on for >= 2^24 entries only)
    "warp_order_keys": dict(warp_order=1),
    "warp_order_keys_small_packs": dict(warp_order=1, warp_max_out_degree=12, warp_area_ints=144, chunk=7),
    "warp_order_vertex": dict(warp_order=2),
}


@pytest.mark.parametrize("name", sorted(PARAM_SETS))
def test_param_regimes(T, name):
    gs = [G.rmat(14, 16, seed=13), G.complete(300), G.rgg(30_000, 40.0, seed=14)]
    with T.Context(0, params=PARAM_SETS[name]) as c:
        for g in gs:
            assert gpu_count(c, g) == oracle.count(g), (name, g.name)


# thread-block shapes whose tables reach 2^12 and 2^13 buckets: with 100 KB
# blocks a part holds up to 4096 keys, with 200 KB up to 8192, and the
# signature probe is compiled once per table size (2^6 .. 2^13 buckets)
BLOCK_SHAPES = {
    "default": {},
    "blocks_100k": dict(block_threads=512, block_smem_bytes=100 * 1024, item_neighbors=512),
    "blocks_200k": dict(block_threads=1024, block_smem_bytes=200 * 1024, item_neighbors=1024),
}


@pytest.mark.parametrize("shape", sorted(BLOCK_SHAPES))
def test_block_table_sizes(T, shape):
    # K_2100: vertex i keeps the 2099 - i larger ids, so the thread-block tables
    # run through every size from 2^6 buckets up to the shape's largest part
    k = G.complete(2100)
    g = G.rmat(14, 16, seed=17)
    with T.Context(0, params=BLOCK_SHAPES[shape]) as c:
        assert gpu_count(c, k) == math.comb(2100, 3)
        assert gpu_count(c, g) == oracle.count(g)


def _bucket_collision_graph(k, stride=1024):
    # u = 0 joined to k vertices whose ids are multiples of `stride`, which form
    # a clique: every key of N+(0) hashes to bucket 0 for any B <= stride.
    hub = [stride * (i + 1) for i in range(k)]
    n = stride * (k + 1) + 1
    e = [(0, h) for h in hub] + [(a, b) for i, a in enumerate(hub) for b in hub[i + 1:]]
    return G.from_edge_list(n, e)


@pytest.mark.parametrize("k,params", [(60, {}), (300, {}), (200, dict(warp_max_out_degree=255, warp_area_ints=2304)),
                                      (600, {}), (500, dict(block_threads=64, block_smem_bytes=8192,
                                                             item_neighbors=64))])
@pytest.mark.parametrize("hash_mode", [1, 0])
def test_adversarial_overflow(T, k, params, hash_mode):
    # with Algorithm 1's hash (x mod B, hash_mode 1) every key of N+(0) lands in
    # bucket 0 and the overflow chains run through hundreds of buckets
    g = _bucket_collision_graph(k)
    want = math.comb(k, 2) + math.comb(k, 3)
    assert oracle.count(g) == want
    with T.Context(0, params=dict(params, hash_mode=hash_mode)) as c:
        assert gpu_count(c, g) == want


@pytest.mark.parametrize("warp_order", [0, 1])
def test_shards_sum_to_total(T, warp_order):
    g = G.rmat(13, 16, seed=15)
    want = oracle.count(g)
    parts = []
    for i in range(3):
        with T.Context(0, params=dict(shard_count=3, shard_index=i, warp_order=warp_order)) as c:
            parts.append(gpu_count(c, g))
    assert sum(parts) == want and all(p > 0 for p in parts)


def test_ordered_warp_list_launches_and_host_pieces(T):
    # warp_order 1: binning gives every warp-class vertex a locality key and
    # becomes histogram + 3 scan kernels + placement (4 more launches), and the
    # thread-block work items are ordered by key too (item keys + 3 scan
    # kernels + placement: 5 more); the piecewise host path (>= 2^20 entries)
    # takes the same order
    g = G.rmat(13, 16, seed=20)
    big = G.disjoint_union([G.rgg(30_001, 40.0, seed=35), G.star(5000), G.wheel(700),
                            G.rmat(14, 16, seed=36), G.complete(45)])
    with T.Context(0, params=dict(warp_order=1)) as c:
        rp, col = dev(g)
        l0 = c.kernel_launches()
        assert c.count(g.n, rp, col) == oracle.count(g)
        assert c.kernel_launches() - l0 == 17
        assert gpu_count(c, G.shuffle_rows(g, 3)) == oracle.count(g)   # unsorted rows: an arbitrary order
        # a compact DAG (tc_orient) counted with the ordered list, per vertex
        d = c.orient(g.n, rp, col)
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        l1 = c.kernel_launches()
        want_total, want_pv = oracle.count_dag(oracle.orient(g), per_vertex=True)
        assert c.count_dag(d, per_vertex=pv) == want_total
        assert c.kernel_launches() - l1 == 13     # ordered binning (5) + item ordering (5) + 3 counting
        assert np.array_equal(pv.cpu().numpy().astype(np.uint64), want_pv)
        d.free()
        want = oracle.count(big)
        for bits in (32, 64):
            rph = np.ascontiguousarray(big.row_ptr.astype(np.int64 if bits == 64 else np.int32))
            colh = np.ascontiguousarray(big.col, dtype=np.int32)
            assert c.count_host(big.n, rph, colh) == want
            assert c.count_host(big.n, torch.from_numpy(rph).pin_memory().numpy(),
                                torch.from_numpy(colh).pin_memory().numpy()) == want


# ------------------------------------------------------------ entry points

def test_count_async_and_host(ctx):
    g = G.rmat(12, 16, seed=16)
    want = oracle.count(g)
    rp, col = dev(g)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ctx.count_async(g.n, rp, col, out, err)
    torch.cuda.synchronize()
    assert int(out.item()) == want and int(err.item()) == 0
    assert ctx.count_host(g.n, g.row_ptr, g.col) == want
    assert ctx.count_host(g.n, g.row_ptr.astype(np.int32), g.col) == want


def test_repeated_calls_are_identical(ctx):
    g = G.rmat(14, 16, seed=17)
    rp, col = dev(g)
    vals = {ctx.count(g.n, rp, col) for _ in range(5)}
    assert vals == {oracle.count(g)}


# ------------------------------------------------------------- bad inputs

def test_bad_column_id(T, ctx):
    g = G.rmat(10, 8, seed=18)
    col = g.col.copy()
    col[17] = g.n + 5
    rp, c = dev(G.Csr(g.n, g.row_ptr, col))
    with pytest.raises(T.TcError) as ei:
        ctx.count(g.n, rp, c)
    assert ei.value.status == T.TC_ERR_BAD_GRAPH
    col[17] = -3
    rp, c = dev(G.Csr(g.n, g.row_ptr, col))
    with pytest.raises(T.TcError):
        ctx.count(g.n, rp, c)
    # the context stays usable
    assert gpu_count(ctx, g) == oracle.count(g)


def test_bad_row_ptr(T, ctx):
    g = G.rmat(10, 8, seed=19)
    rp = g.row_ptr.copy()
    rp[100] = rp[101] + 5        # not monotone
    with pytest.raises(T.TcError) as ei:
        ctx.count(g.n, *dev(G.Csr(g.n, rp, g.col)))
    assert ei.value.status == T.TC_ERR_BAD_GRAPH
    rp = g.row_ptr.copy()
    rp[-1] = rp[-1] + 1000       # beyond nnz
    with pytest.raises(T.TcError):
        ctx.count(g.n, *dev(G.Csr(g.n, rp, g.col)))


def test_asymmetric_input_does_not_overflow(T, ctx):
    # Every row has 10 entries (forward ids, padded with self-loops), so all
    # degrees tie and every forward entry is kept: m would exceed nnz/2.
    n, d = 1000, 10
    rows = [[v if v < n else u for v in range(u + 1, u + 1 + d)] for u in range(n)]
    rp = np.arange(0, n * d + 1, d, dtype=np.int64)
    col = np.array(rows, dtype=np.int32).ravel()
    with pytest.raises(T.TcError) as ei:
        ctx.count(n, *dev(G.Csr(n, rp, col)))
    assert ei.value.status == T.TC_ERR_BAD_GRAPH
    assert gpu_count(ctx, G.complete(10)) == 120


def test_invalid_params(T):
    for bad in (dict(warp_min_buckets=48), dict(item_neighbors=2048), dict(shard_count=2, shard_index=2),
                dict(warp_max_out_degree=256), dict(block_threads=100), dict(chunk=33), dict(warp_area_ints=320),
                dict(warp_min_buckets=8), dict(hash_mode=2), dict(balance=5), dict(balance=-1),
                dict(balance=1, hash_mode=1), dict(warp_order=3), dict(warp_order=-1)):
        with pytest.raises(T.TcError) as ei:
            T.Context(0, params=bad)
        assert ei.value.status == T.TC_ERR_INVALID_ARG


def test_phase_timing_and_launch_count(T):
    g = G.rmat(13, 16, seed=20)
    with T.Context(0, params=dict(record_timing=1)) as c:
        rp, col = dev(g)
        l0 = c.kernel_launches()
        assert c.count(g.n, rp, col) == oracle.count(g)
        # row-local DAG: degree + 2 orientation count kernels, bin, 3 counting (block
        # workers, quad and octet builds of the warp workers), finish
        assert c.kernel_launches() - l0 == 8
        d = c.orient(g.n, rp, col)              # a compact DAG: 8 orientation kernels
        l1 = c.kernel_launches()
        assert c.count_dag(d) == oracle.count(g)
        assert c.kernel_launches() - l1 == 4     # bin + 3 counting
        d.free()
        t = c.read_timing()
        assert t["calls"] == 2 and t["orient_ms"] > 0 and t["count_ms"] > 0
        assert c.read_timing()["calls"] == 0


def test_build_probe_cycle_split(T):
    # record_timing = 2: the workers' cycles in table builds and in probes. The
    # edge-centric ablation rebuilds N+(u)'s table once per out-edge, so its
    # build share must exceed the vertex-centric one (Sec. 3.3).
    g = G.rmat(14, 16, seed=23)
    shares = {}
    for ec in (0, 1):
        with T.Context(0, params=dict(record_timing=2, edge_centric=ec)) as c:
            assert gpu_count(c, g) == oracle.count(g)
            t = c.read_timing()
            assert t["build_cycles"] > 0 and t["probe_cycles"] > 0
            shares[ec] = t["build_cycles"] / (t["build_cycles"] + t["probe_cycles"])
            assert c.read_timing()["build_cycles"] == 0      # reading starts a new period
    assert shares[1] > shares[0]


def test_host_csr_pinned_and_pageable(ctx):
    # tc_count_host from pageable and pinned host arrays; graphs of 2^20 or more
    # entries are copied in row pieces that are oriented as they land (the last
    # graph, with hub, mid and ragged rows), smaller ones in one copy
    gs = [G.disjoint_union([G.star(3000), G.complete(300), G.rmat(12, 16, seed=33)]),
          G.rgg(20_000, 30.0, seed=34), G.empty(9), G.complete(3),
          G.disjoint_union([G.rgg(30_001, 40.0, seed=35), G.star(5000), G.wheel(700),
                            G.rmat(14, 16, seed=36), G.complete(45)])]
    for g in gs:
        want = oracle.count(g)
        for bits in (32, 64):
            rp = np.ascontiguousarray(g.row_ptr.astype(np.int64 if bits == 64 else np.int32))
            col = np.ascontiguousarray(g.col, dtype=np.int32)
            assert ctx.count_host(g.n, rp, col) == want
            rp_pin = torch.from_numpy(rp).pin_memory()
            col_pin = torch.from_numpy(col).pin_memory()
            assert col_pin.is_pinned() or g.nnz == 0
            assert ctx.count_host(g.n, rp_pin.numpy(), col_pin.numpy()) == want
            assert ctx.count_host(g.n, rp_pin.numpy(), col_pin.numpy()) == want  # reuse the device copy
