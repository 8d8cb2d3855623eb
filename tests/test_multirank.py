"""The multi-rank path on CPU: gloo process groups of 2 and 3 ranks.

Each rank counts the apexes u with u % world == rank (the oracle's per-vertex
counts stand in for the kernels, which apply the same rule through
tc_params.shard_count / shard_index), then the ranks exchange one 64-bit sum
and one max of their times through paper_2103_08053_gb300.shard.combine, as
bench.py does over NCCL. The sum must equal the whole count on every rank.
"""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as ge
    ge._load_builder().build()


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, graph_args):
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np

    import graphgen as G
    import oracle
    from paper_2103_08053_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = G.rmat(*graph_args)
        od = oracle.orient(g)
        mine = np.array([u for u in range(g.n) if shard.owns(u, rank, world)], dtype=np.int64)
        part = int(oracle.count_dag_at(od, mine).sum()) if mine.size else 0
        total, ms = shard.combine(part, float(rank + 1))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"part": part, "total": total, "ms": ms, "owned": int(mine.size)}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_counts_sum_to_the_whole(built, tmp_path, world):
    import graphgen as G
    import oracle
    graph_args = (11, 12, 17)  # R-MAT scale 11, edge factor 12, seed 17
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path), graph_args), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    g = G.rmat(*graph_args)
    want = oracle.count(g)
    assert want > 0
    assert sum(r["part"] for r in res) == want
    assert all(r["total"] == want for r in res)          # every rank sees the sum
    assert all(r["ms"] == float(world) for r in res)     # and the slowest rank's time
    assert sum(r["owned"] for r in res) == g.n           # the rule covers every vertex once
    assert all(r["part"] > 0 for r in res)


def test_shard_rule_and_identity_without_a_group(built):
    from paper_2103_08053_gb300 import shard
    assert shard.shard_params(1, 4) == {"shard_count": 4, "shard_index": 1}
    for bad in ((4, 4), (-1, 2), (0, 0)):
        with pytest.raises(ValueError):
            shard.shard_params(*bad)
    assert [u for u in range(10) if shard.owns(u, 2, 3)] == [2, 5, 8]
    assert not dist.is_initialized()
    assert shard.combine(123, 4.5) == (123, 4.5)
