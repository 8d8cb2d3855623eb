"""tc_count_dag_noalloc, the entry point for callers that cannot allocate
device memory (their GPU memory is held by another allocator, or they must not
risk the device-wide synchronisation a cudaMalloc can cause). It is checked
through the C ABI against tc_count_dag on two calls in a row that share its
static scratch array. Counts are integers: the outputs must be equal.

This file is collected last on purpose; it works both alone in a fresh process
(the first call sets the device up) and after every other test.
"""
import ctypes

import numpy as np
import pytest

import graphgen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as ge
    ge._load_builder().build()
    import paper_2103_08053_gb300 as T
    return T


def _device_dag(ctx, g):
    d = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).to(d)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d)
    return ctx.orient(g.n, rp, col)


def test_noalloc_equals_count_dag_on_two_calls_in_a_row(T):
    from paper_2103_08053_gb300 import _tc
    # the second graph has thread-block vertices (K_300: d+ up to 299) and the
    # first only warp vertices, so the second call must not see the first's state
    graphs = [G.rmat(14, 16, seed=33), G.disjoint_union([G.complete(300), G.rmat(12, 8, seed=34)])]
    with T.Context(0) as ctx:
        dags = [_device_dag(ctx, g) for g in graphs]
        want = [ctx.count_dag(d) for d in dags]
        out = torch.zeros(len(dags), dtype=torch.int64, device="cuda")
        err = torch.full((len(dags),), -1, dtype=torch.int32, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for i, d in enumerate(dags):
            st = _tc.tc_count_dag_noalloc(ctypes.byref(d.raw), ctypes.c_void_p(out.data_ptr() + 8 * i),
                                          ctypes.c_void_p(err.data_ptr() + 4 * i), stream)
            assert st == T.TC_OK, _tc.tc_last_error(None)
        torch.cuda.synchronize()
        assert out.cpu().tolist() == want
        assert err.cpu().tolist() == [0, 0]
        assert want[1] >= 4455100  # C(300,3) alone
        for d in dags:
            d.free()


def test_noalloc_rejects_graphs_beyond_its_scratch(T):
    from paper_2103_08053_gb300 import _tc
    big = _tc.tc_dag(1 << 20, 10, 1, 1)  # n over the limit; the pointers are never used
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = _tc.tc_count_dag_noalloc(ctypes.byref(big), ctypes.c_void_p(out.data_ptr()), None, None)
    assert st == T.TC_ERR_UNSUPPORTED
    assert b"static scratch" in _tc.tc_last_error(None)
