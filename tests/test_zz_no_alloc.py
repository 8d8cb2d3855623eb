"""tc_count_dag_noalloc, the entry point for callers that cannot allocate
device memory (their GPU memory is held by another allocator, or they must not
risk the device-wide synchronisation a cudaMalloc can cause). It is checked
through the C ABI against the CPU oracle and against tc_count_dag on two calls
in a row that share its static scratch array, on a count above 2^32 against
the closed form C(n, 3), and beside contexts whose thread-block workers use
other shared-memory sizes (the kernels' launch limits are shared by all
callers in the process). Counts are integers: the outputs must be equal.

This file is collected last on purpose; it works both alone in a fresh process
(the first call sets the device up) and after every other test.
"""
import ctypes
from math import comb

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


def _dev(g):
    d = torch.device("cuda", 0)
    return (g.n, torch.from_numpy(g.row_ptr.astype(np.int32)).to(d),
            torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d))


def _noalloc(T, dags):
    """One tc_count_dag_noalloc call per DAG, in a row on the current stream."""
    from paper_2103_08053_gb300 import _tc
    out = torch.zeros(len(dags), dtype=torch.int64, device="cuda")
    err = torch.full((len(dags),), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for i, d in enumerate(dags):
        st = _tc.tc_count_dag_noalloc(ctypes.byref(d.raw), ctypes.c_void_p(out.data_ptr() + 8 * i),
                                      ctypes.c_void_p(err.data_ptr() + 4 * i), stream)
        assert st == T.TC_OK, _tc.tc_last_error(None)
    torch.cuda.synchronize()
    return [int(x) & (2 ** 64 - 1) for x in out.cpu().tolist()], err.cpu().tolist()


def test_noalloc_equals_oracle_and_count_dag_on_two_calls_in_a_row(T):
    # the second graph has thread-block vertices (K_300: d+ up to 299) and the
    # first only warp vertices, so the second call must not see the first's state
    graphs = [G.rmat(14, 16, seed=33), G.disjoint_union([G.complete(300), G.rmat(12, 8, seed=34)])]
    want = [oracle.count_dag(oracle.orient(g)) for g in graphs]
    with T.Context(0) as ctx:
        dags = [ctx.orient(*_dev(g)) for g in graphs]
        assert [ctx.count_dag(d) for d in dags] == want
        got, err = _noalloc(T, dags)
        assert got == want
        assert err == [0, 0]
        assert want[1] >= comb(300, 3)
        for d in dags:
            d.free()


def test_noalloc_count_above_2_to_the_32(T):
    g = G.complete(3000)
    with T.Context(0) as ctx:
        dag = ctx.orient(*_dev(g))
        got, err = _noalloc(T, [dag, dag])
        assert got == [comb(3000, 3)] * 2 and err == [0, 0]
        dag.free()


@pytest.mark.parametrize("order", ["context_first", "noalloc_first"])
def test_noalloc_beside_contexts_with_other_block_shapes(T, order):
    # the counting kernels' dynamic shared-memory limits are per device and
    # shared by every caller: a context with 200 KB thread-block workers, one
    # with smaller tables and the allocation-free entry point (default shapes)
    # must all keep launching, whichever sets its limits first
    g = G.disjoint_union([G.complete(400), G.rmat(13, 16, seed=35)])
    want = oracle.count(g)
    big = dict(block_threads=1024, block_smem_bytes=200 * 1024, item_neighbors=1024)
    small = dict(block_threads=128, block_smem_bytes=16 * 1024, item_neighbors=128, warp_area_ints=576,
                 warp_max_out_degree=64)
    n, rp, col = _dev(g)
    with T.Context(0) as base:
        dag = base.orient(n, rp, col)
        if order == "noalloc_first":
            assert _noalloc(T, [dag])[0] == [want]
        with T.Context(0, params=big) as cb, T.Context(0, params=small) as cs:
            for _ in range(2):
                assert cb.count(n, rp, col) == want
                assert _noalloc(T, [dag])[0] == [want]
                assert cs.count(n, rp, col) == want
                assert cb.count(n, rp, col) == want
        assert base.count_dag(dag) == want
        dag.free()


def test_noalloc_rejects_graphs_beyond_its_scratch(T):
    from paper_2103_08053_gb300 import _tc
    big = _tc.tc_dag(1 << 20, 10, 1, 1)  # n over the limit; the pointers are never used
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = _tc.tc_count_dag_noalloc(ctypes.byref(big), ctypes.c_void_p(out.data_ptr()), None, None)
    assert st == T.TC_ERR_UNSUPPORTED
    assert b"static scratch" in _tc.tc_last_error(None)
