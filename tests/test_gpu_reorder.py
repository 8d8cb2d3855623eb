"""tc_reorder (Sec. 4.1) vs the oracle's sequential definitions: new ids
bit-exact, the relabelled CSR entry for entry, and the count unchanged."""
import numpy as np
import pytest

import graphgen as G
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = [oracle.REORDER_INDEGREE, oracle.REORDER_COLLECTIVE]


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as ge
    ge._load_builder().build()
    import paper_2103_08053_gb300 as T
    return T


def dev(g, bits=32):
    d = torch.device("cuda", 0)
    rp = torch.from_numpy(np.asarray(g.row_ptr).astype(np.int64 if bits == 64 else np.int32)).to(d)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d)
    return g.n, rp, col


def check(T, c, g, kind, bits=32):
    n, rp, col = dev(g, bits)
    nid, rp2, col2 = c.reorder(n, rp, col, kind)
    want = oracle.reorder(g, kind)
    assert np.array_equal(nid.cpu().numpy(), want)
    h = oracle.relabel(g, want)
    assert np.array_equal(rp2.cpu().numpy().astype(np.int64), h.row_ptr)
    assert np.array_equal(col2.cpu().numpy(), h.col)
    assert c.count(n, rp2, col2) == c.count(n, rp, col) == oracle.count(g)


def graphs():
    yield G.complete(40)
    yield G.star(3000)
    yield G.wheel(33)
    yield G.friendship(700)
    yield G.cycle(5)
    yield G.empty(7)
    yield G.complete(1)
    yield G.rgg(6000, 18.0, seed=4)
    for s in range(3):
        yield G.rmat(12 + s, 8, seed=400 + s)   # several radix tiles, ragged tail
    yield G.erdos_renyi(5000, 0.004, seed=41)


@pytest.mark.parametrize("kind", KINDS)
def test_reorder_matches_oracle(T, kind):
    with T.Context(0) as c:
        for g in graphs():
            check(T, c, g, kind)


@pytest.mark.parametrize("kind", KINDS)
def test_reorder_int64_offsets(T, kind):
    with T.Context(0) as c:
        check(T, c, G.rmat(11, 12, seed=77), kind, bits=64)


def test_reorder_new_id_only_and_bad_arguments(T):
    g = G.rmat(10, 8, seed=5)
    with T.Context(0) as c:
        n, rp, col = dev(g)
        nid = c.reorder(n, rp, col, T.TC_REORDER_COLLECTIVE, relabel=False)
        assert np.array_equal(nid.cpu().numpy(), oracle.reorder(g, 2))
        with pytest.raises(T.TcError) as ei:
            c.reorder(n, rp, col, 3)
        assert ei.value.status == T.TC_ERR_INVALID_ARG
        # the context stays usable
        assert c.count(n, rp, col) == oracle.count(g)
        assert c.reorder(0, torch.zeros(1, dtype=torch.int32, device="cuda"),
                         torch.zeros(0, dtype=torch.int32, device="cuda"), 1, relabel=False).numel() == 0


@pytest.mark.slow
def test_reorder_rmat16_workload(T):
    g = G.workload("rmat16")
    with T.Context(0) as c:
        for kind in KINDS:
            check(T, c, g, kind)


@pytest.mark.parametrize("seed", range(3))
def test_collision_statistics_match_oracle(T, seed):
    g = G.rmat(11, 8, seed=500 + seed)
    with T.Context(0) as c:
        for kind in (None, *KINDS):
            h = g if kind is None else oracle.relabel(g, oracle.reorder(g, kind))
            d = c.orient(*dev(h))
            st = c.dag_stats(d)
            d.free()
            od = oracle.orient(h)
            assert (st["max_collision_mod32"], st["phi_mod32"]) == oracle.collision_stats(od, "mod32")
            assert (st["max_collision_mult32"], st["phi_mult32"]) == oracle.collision_stats(od, "mult32")
