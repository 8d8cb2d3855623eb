"""Counts above 2^32 (Algorithm 1's count += carried in 64 bits).

The complete graph K_3000 has C(3000, 3) = 4,495,501,000 > 2^32 triangles: a
closed form, independent of the oracle and of the GPU path. Every counting
entry point must return it exactly; a 32-bit accumulator anywhere on the path
(per-lane hits, warp or block partials, the final total, a per-graph batch sum)
would wrap to 200,533,704. K_3000 also exercises the thread-block workers'
split tables: after orientation by (degree, id) vertex i has d+ = 2999 - i,
and the out-lists of the lowest ids are longer than one table part.
"""
from math import comb

import numpy as np
import pytest

import graphgen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 3000
WANT = comb(N, 3)
assert WANT == 4_495_501_000 and WANT > 2 ** 32


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as ge
    ge._load_builder().build()
    import paper_2103_08053_gb300 as T
    return T


@pytest.fixture(scope="module")
def k3000():
    return G.complete(N)


def dev(g, bits=32):
    d = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int64 if bits == 64 else np.int32)).to(d)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(d)
    return g.n, rp, col


@pytest.mark.parametrize("bits", [32, 64])
def test_count_and_count_async(T, k3000, bits):
    with T.Context(0) as c:
        n, rp, col = dev(k3000, bits)
        assert c.count(n, rp, col) == WANT
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        c.count_async(n, rp, col, out, err)
        torch.cuda.synchronize()
        assert int(out.item()) & (2 ** 64 - 1) == WANT and int(err.item()) == 0


def test_count_host(T, k3000):
    with T.Context(0) as c:
        assert c.count_host(k3000.n, k3000.row_ptr.astype(np.int32),
                            np.ascontiguousarray(k3000.col, dtype=np.int32)) == WANT


def test_count_batch_two_copies(T, k3000):
    with T.Context(0) as c:
        g = dev(k3000)
        small = dev(G.complete(10))
        assert c.count_batch([g, small, g]) == [WANT, comb(10, 3), WANT]


def test_count_dag_total_and_per_vertex(T, k3000):
    with T.Context(0) as c:
        dag = c.orient(*dev(k3000))
        assert dag.m == comb(N, 2)
        pv = torch.zeros(N, dtype=torch.int64, device="cuda")
        assert c.count_dag(dag, per_vertex=pv) == WANT
        # apex(i) = C(2999 - i, 2): vertex i precedes exactly the 2999 - i higher ids
        got = pv.cpu().numpy().astype(np.uint64)
        want = np.array([comb(N - 1 - i, 2) for i in range(N)], dtype=np.uint64)
        assert np.array_equal(got, want)
        dag.free()

