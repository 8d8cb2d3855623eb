"""Device allocation failures, injected on the host with tc_inject_oom.

The failing allocation is never attempted: the library returns TC_ERR_OOM as
if cudaMalloc had reported an out-of-memory device, so nothing faults or
hangs on the GPU. Each entry point that allocates must report the status and
leave its context usable: the next call on the same context allocates again
and gives the oracle's count.
"""
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


def dev(g):
    d = torch.device("cuda", 0)
    return (g.n, torch.from_numpy(g.row_ptr.astype(np.int32)).to(d),
            torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d))


@pytest.mark.parametrize("nth", [1, 2, 3, 5])
def test_count_reports_oom_then_counts(T, nth):
    g = G.rmat(12, 16, seed=41)
    want = oracle.count(g)
    n, rp, col = dev(g)
    with T.Context(0) as c:  # fresh context: its first count grows the workspace
        c.inject_oom(nth)
        with pytest.raises(T.TcError) as e:
            c.count(n, rp, col)
        assert e.value.status == T.TC_ERR_OOM
        assert b"injected" in T._tc.tc_last_error(c.handle)
        assert c.count(n, rp, col) == want
        assert c.count(n, rp, col) == want


def test_host_and_dag_entry_points_report_oom(T):
    g = G.rmat(11, 8, seed=42)
    want = oracle.count(g)
    n, rp, col = dev(g)
    with T.Context(0) as c:
        c.inject_oom(1)
        with pytest.raises(T.TcError) as e:
            c.count_host(g.n, g.row_ptr.astype(np.int32), np.ascontiguousarray(g.col, dtype=np.int32))
        assert e.value.status == T.TC_ERR_OOM
        assert c.count_host(g.n, g.row_ptr.astype(np.int32), np.ascontiguousarray(g.col, dtype=np.int32)) == want
    with T.Context(0) as c:
        dag = c.orient(n, rp, col)  # grows the workspace
        c.inject_oom(1)              # tc_orient's own DAG arrays
        with pytest.raises(T.TcError) as e:
            c.orient(n, rp, col)
        assert e.value.status == T.TC_ERR_OOM
        assert c.count_dag(dag) == want
        dag.free()


def test_batch_reports_oom_then_counts(T):
    gs = [G.batch_graph(7, i) for i in range(24)]
    want = [oracle.count(g) for g in gs]
    tensors = [dev(g) for g in gs]
    with T.Context(0) as c:
        c.inject_oom(1)
        with pytest.raises(T.TcError) as e:
            c.count_batch(tensors)
        assert e.value.status == T.TC_ERR_OOM
        assert c.count_batch(tensors) == want


def test_submit_reports_oom_then_serves(T):
    gs = [G.batch_graph(8, i) for i in range(6)]
    want = [oracle.count(g) for g in gs]
    host = [(g.n, g.row_ptr.astype(np.int32), np.ascontiguousarray(g.col, dtype=np.int32)) for g in gs]
    with T.Context(0, mem_budget=1 << 28) as c:
        c.inject_oom(1)  # the serving arena, allocated by the first submission
        with pytest.raises(T.TcError) as e:
            c.submit(*host[0])
        assert e.value.status == T.TC_ERR_OOM
        tickets = [c.submit(*h) for h in host]
        c.drain()
        assert [c.poll(t) for t in tickets] == want
        # a failure inside a running round: the next round's workspace growth
        big = G.rmat(14, 16, seed=43)
        c.inject_oom(1)
        t = c.submit(big.n, big.row_ptr.astype(np.int32), np.ascontiguousarray(big.col, dtype=np.int32))
        c.drain()
        got = None
        try:
            got = c.poll(t)
        except T.TcError as err:
            assert err.status == T.TC_ERR_OOM
        if got is not None:  # the round fitted the workspace already: no allocation was needed
            assert got == oracle.count(big)
        c.inject_oom(0)
        t = c.submit(big.n, big.row_ptr.astype(np.int32), np.ascontiguousarray(big.col, dtype=np.int32))
        c.drain()
        assert c.poll(t) == oracle.count(big)


def test_inject_oom_rejects_bad_arguments(T):
    assert T._tc.tc_inject_oom(None, 1) == T.TC_ERR_INVALID_ARG
    with T.Context(0) as c:
        assert T._tc.tc_inject_oom(c.handle, -1) == T.TC_ERR_INVALID_ARG
