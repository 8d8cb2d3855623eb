"""tc_count_batch vs the CPU oracle, graph by graph (bit-exact)."""
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


def dev(g, bits=32):
    d = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int64 if bits == 64 else np.int32)).to(d)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d)
    return g.n, rp, col


def mixed_graphs(seed):
    rng = np.random.default_rng(seed)
    gs = [G.complete(40), G.empty(0), G.cycle(3), G.wheel(33), G.empty(5), G.complete(300),
          G.star(1000), G.rgg(3000, 20.0, seed=seed)]
    for i in range(12):
        gs.append(G.rmat(int(rng.integers(6, 12)), int(rng.integers(2, 17)), seed=seed * 100 + i))
    gs += [G.batch_graph(seed, i) for i in range(6)]
    return gs


def test_batch_matches_oracle_per_graph(T):
    gs = mixed_graphs(1)
    want = [oracle.count(g) for g in gs]
    with T.Context(0) as c:
        tensors = [dev(g) for g in gs]
        assert c.count_batch(tensors) == want
        # the per-graph path agrees too
        assert [c.count(n, rp, col) for n, rp, col in tensors] == want


def test_batch_replay_with_new_graphs_of_the_same_shape(T):
    # relabelled copies keep every n and nnz, so the second and third calls
    # replay the captured CUDA graph with new descriptors and new edges
    a = [G.erdos_renyi(500, 0.05, seed=s) for s in range(20)]
    b = [G.shuffle_rows(G.relabel(g, np.random.default_rng(s).permutation(g.n)), s) for s, g in enumerate(a)]
    with T.Context(0) as c:
        for batch in (a, b, a, b):
            want = [oracle.count(g) for g in batch]
            assert c.count_batch([dev(g) for g in batch]) == want
        l0 = c.kernel_launches()
        c.count_batch([dev(g) for g in a])
        # 3 orientation + bin + 3 counting (block workers, the quad and the octet
        # builds of the warp workers) + segsum, replayed
        assert c.kernel_launches() - l0 == 8


def test_batch_int64_offsets_and_block_vertices(T):
    gs = [G.complete(260), G.rmat(13, 16, seed=5), G.friendship(500)]
    want = [oracle.count(g) for g in gs]
    with T.Context(0, params=dict(warp_max_out_degree=64, item_neighbors=64)) as c:
        assert c.count_batch([dev(g, 64) for g in gs]) == want


def test_batch_errors(T):
    with T.Context(0) as c:
        with pytest.raises(T.TcError) as ei:
            c.count_batch([dev(G.complete(5)), dev(G.complete(6), 64)])
        assert ei.value.status == T.TC_ERR_UNSUPPORTED
        bad = G.rmat(8, 4, seed=3)
        col = bad.col.copy()
        col[3] = bad.n + 7
        with pytest.raises(T.TcError) as ei:
            c.count_batch([dev(G.complete(5)), dev(G.Csr(bad.n, bad.row_ptr, col))])
        assert ei.value.status == T.TC_ERR_BAD_GRAPH
        assert c.count_batch([dev(G.complete(7))]) == [35]
        assert c.count_batch([]) == []


def test_batched_workload_sample(T):
    gs = [G.batch_graph(4, i) for i in range(64)]
    want = [oracle.count(g) for g in gs]
    with T.Context(0) as c:
        assert c.count_batch([dev(g) for g in gs]) == want


def test_autotune_keeps_counts_and_caches(T, tmp_path):
    gs = [G.batch_graph(31, i) for i in range(48)]
    want = [oracle.count(g) for g in gs]
    cache = str(tmp_path / "tune.txt")
    with T.Context(0) as c:
        tensors = [dev(g) for g in gs]
        best = c.autotune(tensors, cache_path=cache)
        assert c.get_params()["warp_max_out_degree"] == best["warp_max_out_degree"]
        assert c.count_batch(tensors) == want
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("sig ")
    with T.Context(0) as c:            # the second tuner reads the cache
        again = c.autotune([dev(g) for g in gs], cache_path=cache)
        assert again == best
        assert c.count_batch([dev(g) for g in gs]) == want
    assert len(open(cache).read().splitlines()) == 1
    with T.Context(0) as c:            # one graph: tuned with tc_count
        g = G.rmat(14, 16, seed=32)
        c.autotune([dev(g)])
        assert c.count(*dev(g)) == oracle.count(g)
