"""Serving (tc_submit / tc_poll): continuous batching under a memory budget.
Every result must equal the oracle's count of its own graph, alone or in a mix."""
import threading
import time

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


def host(g, bits=32):
    return g.n, g.row_ptr.astype(np.int64 if bits == 64 else np.int32), np.ascontiguousarray(g.col, dtype=np.int32)


def wait_all(c, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                v = c.poll(t)
                if v is not None:
                    out[t] = v
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.001)
    return [out[t] for t in tickets]


def test_serve_mixed_requests(T):
    gs = [G.batch_graph(7, i) for i in range(40)] + [G.complete(200), G.empty(3), G.rmat(14, 16, seed=8)]
    want = [oracle.count(g) for g in gs]
    with T.Context(0, mem_budget=1 << 30) as c:
        tickets = [c.submit(*host(g)) for g in gs]
        assert wait_all(c, tickets) == want


def test_alone_equals_in_the_mix(T):
    x = G.rmat(13, 16, seed=11)
    want = oracle.count(x)
    with T.Context(0, mem_budget=1 << 30) as c:
        alone = wait_all(c, [c.submit(*host(x))])[0]
        others = [G.batch_graph(12, i) for i in range(60)]
        tickets = [c.submit(*host(g)) for g in others[:30]]
        tx = c.submit(*host(x))
        tickets += [c.submit(*host(g)) for g in others[30:]]
        res = wait_all(c, tickets + [tx])
        assert alone == res[-1] == want
        assert res[:-1] == [oracle.count(g) for g in others]


def test_tight_budget_admits_as_memory_frees(T):
    gs = [G.erdos_renyi(4000, 0.01, seed=s) for s in range(24)]
    want = [oracle.count(g) for g in gs]
    one = gs[0].nnz * 4 + (gs[0].n + 1) * 4
    with T.Context(0, mem_budget=3 * one + 8192) as c:   # room for about two requests at a time
        tickets = [c.submit(*host(g)) for g in gs]
        c.drain()
        assert wait_all(c, tickets) == want


def test_concurrent_submitters(T):
    gs = [G.batch_graph(13, i) for i in range(48)]
    want = {i: oracle.count(g) for i, g in enumerate(gs)}
    got = {}
    with T.Context(0, mem_budget=1 << 30) as c:
        def client(lo, hi):
            ts = {i: c.submit(*host(gs[i], 64 if i % 2 else 32)) for i in range(lo, hi)}
            for i, t in ts.items():
                while (v := c.poll(t)) is None:
                    time.sleep(0.0005)
                got[i] = v
        th = [threading.Thread(target=client, args=(k * 12, k * 12 + 12)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    assert got == want


def test_serve_errors(T):
    with T.Context(0, mem_budget=1 << 20) as c:
        big = G.rmat(14, 16, seed=1)
        with pytest.raises(T.TcError) as ei:
            c.submit(*host(big))
        assert ei.value.status == T.TC_ERR_BUSY
        bad = G.complete(10)
        col = bad.col.copy()
        col[0] = 99
        with pytest.raises(T.TcError) as ei:
            c.submit(bad.n, bad.row_ptr.astype(np.int32), col)
        assert ei.value.status == T.TC_ERR_BAD_GRAPH
        t = c.submit(*host(G.complete(10)))
        assert wait_all(c, [t]) == [120]
        with pytest.raises(T.TcError) as ei:
            c.poll(t)            # retired
        assert ei.value.status == T.TC_ERR_INVALID_ARG
    with T.Context(0) as c:     # no budget: serving is not available
        with pytest.raises(T.TcError) as ei:
            c.submit(*host(G.complete(4)))
        assert ei.value.status == T.TC_ERR_INVALID_ARG


def test_borrowed_submission(T):
    gs = [G.batch_graph(21, i) for i in range(30)] + [G.complete(150)]
    want = [oracle.count(g) for g in gs]
    keep = [host(g, 64 if i % 3 == 0 else 32) for i, g in enumerate(gs)]  # caller keeps these alive
    with T.Context(0, mem_budget=1 << 30) as c:
        tickets = [c.submit_borrowed(*h) for h in keep]
        assert wait_all(c, tickets) == want


def test_large_and_small_classes(T):
    # graphs with more than 2^24 CSR entries run alone in the large slot (low
    # priority, part of the SMs); small ones keep flowing through the others
    big = [G.rmat(20, 16, seed=40 + i) for i in range(2)]
    assert all(g.n + g.nnz > 1 << 24 for g in big)
    small = [G.batch_graph(13, i) for i in range(60)]
    want_big = [oracle.count(g) for g in big]
    want_small = [oracle.count(g) for g in small]
    with T.Context(0, mem_budget=4 << 30) as c:
        tb = [c.submit(*host(g)) for g in big]
        ts = [c.submit(*host(g)) for g in small]
        assert wait_all(c, ts) == want_small
        assert wait_all(c, tb) == want_big
