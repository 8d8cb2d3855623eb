"""CPU oracle for exact triangle counting -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference arm may import this package. The product library
(``paper_2103_08053_gb300``) never imports it, and the two share no code.

``oracle.c`` holds the counting routes (brute force from the definition,
rank-by-degree orientation, node iterator with merge-path intersection);
``alg1.py`` is a plain-Python reading of the paper's Algorithm 1 and its
building blocks. This module wraps the C part with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib_handle = None

I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)
U64P = ctypes.POINTER(ctypes.c_uint64)
U64_MAX = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2, OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.oracle_brute.restype = ctypes.c_uint64
            lib.oracle_brute.argtypes = [ctypes.c_int64, I64P, I32P]
            lib.oracle_orient.restype = ctypes.c_int64
            lib.oracle_orient.argtypes = [ctypes.c_int64, I64P, I32P, I64P, I32P]
            lib.oracle_orient_by_key.restype = ctypes.c_int64
            lib.oracle_orient_by_key.argtypes = [ctypes.c_int64, I64P, I32P, I64P, I64P, I32P]
            lib.oracle_count_dag.restype = ctypes.c_uint64
            lib.oracle_count_dag.argtypes = [ctypes.c_int64, I64P, I32P, U64P, ctypes.c_int]
            lib.oracle_count_dag_at.restype = None
            lib.oracle_count_dag_at.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int64, I64P, U64P,
                                                ctypes.c_int]
            lib.oracle_count.restype = ctypes.c_uint64
            lib.oracle_count.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_reorder.restype = ctypes.c_int
            lib.oracle_reorder.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int, I32P]
            _lib_handle = lib
    return _lib_handle


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.shape[0] == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col


def max_threads() -> int:
    return int(_lib().oracle_max_threads())


def brute(g) -> int:
    """T(G) by the definition (dense triple loop), n <= 4096."""
    rp, col = _csr(g)
    t = _lib().oracle_brute(g.n, rp.ctypes.data_as(I64P), col.ctypes.data_as(I32P))
    if t == U64_MAX:
        raise ValueError("oracle_brute: graph too large")
    return int(t)


class Dag:
    """Oriented graph N+ with sorted rows (int64 offsets, int32 targets)."""

    def __init__(self, n, dag_ptr, dag_col):
        self.n = n
        self.dag_ptr = dag_ptr
        self.dag_col = dag_col

    @property
    def m(self) -> int:
        return int(self.dag_ptr[-1])

    def out_degrees(self) -> np.ndarray:
        return np.diff(self.dag_ptr)


def orient(g, key=None) -> Dag:
    """Rank-by-degree orientation (degree, then id), or by distinct keys."""
    rp, col = _csr(g)
    dag_ptr = np.zeros(g.n + 1, dtype=np.int64)
    dag_col = np.zeros(g.nnz // 2 + 1, dtype=np.int32)
    lib = _lib()
    if key is None:
        m = lib.oracle_orient(g.n, rp.ctypes.data_as(I64P), col.ctypes.data_as(I32P),
                              dag_ptr.ctypes.data_as(I64P), dag_col.ctypes.data_as(I32P))
    else:
        k = np.ascontiguousarray(key, dtype=np.int64)
        if np.unique(k).shape[0] != g.n:
            raise ValueError("orientation keys must be distinct")
        m = lib.oracle_orient_by_key(g.n, rp.ctypes.data_as(I64P), col.ctypes.data_as(I32P),
                                     k.ctypes.data_as(I64P), dag_ptr.ctypes.data_as(I64P),
                                     dag_col.ctypes.data_as(I32P))
    return Dag(g.n, dag_ptr, dag_col[:m])


def _dag_arrays(d: Dag):
    col = d.dag_col if d.dag_col.shape[0] else np.zeros(1, dtype=np.int32)
    return np.ascontiguousarray(d.dag_ptr, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32)


def count_dag(d: Dag, per_vertex: bool = False, threads: int = 0):
    """Node iterator + merge on an oriented graph; optionally apex(u) per u."""
    dp, dc = _dag_arrays(d)
    pv = np.zeros(d.n, dtype=np.uint64) if per_vertex else None
    t = _lib().oracle_count_dag(d.n, dp.ctypes.data_as(I64P), dc.ctypes.data_as(I32P),
                                pv.ctypes.data_as(U64P) if pv is not None else None, threads)
    return (int(t), pv) if per_vertex else int(t)


def count_dag_at(d: Dag, us, threads: int = 0) -> np.ndarray:
    """apex(u) = sum_{v in N+(u)} |N+(u) ∩ N+(v)| for the given vertices."""
    dp, dc = _dag_arrays(d)
    u = np.ascontiguousarray(us, dtype=np.int64)
    out = np.zeros(u.shape[0], dtype=np.uint64)
    _lib().oracle_count_dag_at(d.n, dp.ctypes.data_as(I64P), dc.ctypes.data_as(I32P), u.shape[0],
                               u.ctypes.data_as(I64P), out.ctypes.data_as(U64P), threads)
    return out


def count(g, threads: int = 0) -> int:
    """T(G): orient by (degree, id), then node iterator + merge."""
    rp, col = _csr(g)
    t = _lib().oracle_count(g.n, rp.ctypes.data_as(I64P), col.ctypes.data_as(I32P), threads)
    if t == U64_MAX:
        raise MemoryError("oracle_count: allocation failed")
    return int(t)


def count_many(graphs, workers: int = 0) -> list:
    """T(G) of every graph: one oracle.count per graph, single-threaded each,
    `workers` graphs at a time on host threads (default: all cores)."""
    import concurrent.futures as cf
    workers = workers or os.cpu_count() or 1
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(lambda g: count(g, threads=1), graphs))


REORDER_INDEGREE = 1
REORDER_COLLECTIVE = 2


def reorder(g, kind: int) -> np.ndarray:
    """new_id[old] of the Sec. 4.1 reordering ``kind`` (1: by in-degree in
    N+; 2: neighbours of the largest collective out-degree first), computed on
    the rank-by-degree orientation of g."""
    d = orient(g)
    dp, dc = _dag_arrays(d)
    new_id = np.zeros(max(g.n, 1), dtype=np.int32)
    if _lib().oracle_reorder(g.n, dp.ctypes.data_as(I64P), dc.ctypes.data_as(I32P), int(kind),
                             new_id.ctypes.data_as(I32P)) != 0:
        raise ValueError(f"oracle_reorder failed (kind {kind})")
    return new_id[:g.n]


def relabel(g, new_id):
    """The CSR of g with vertex old renamed new_id[old]: row new_id[u] holds
    new_id[v] for the v of row u, in the same order."""
    from types import SimpleNamespace
    new_id = np.asarray(new_id, dtype=np.int64)
    deg = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
    new_deg = np.zeros(g.n, dtype=np.int64)
    new_deg[new_id] = deg
    rp = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(new_deg, out=rp[1:])
    col = np.zeros(g.nnz, dtype=np.int32)
    src = np.asarray(g.col, dtype=np.int64)
    for u in range(g.n):
        a, b = int(g.row_ptr[u]), int(g.row_ptr[u + 1])
        w = int(rp[new_id[u]])
        col[w:w + (b - a)] = new_id[src[a:b]]
    return SimpleNamespace(n=g.n, nnz=g.nnz, row_ptr=rp, col=col)


def collision_stats(d: Dag, hash_kind: str):
    """(max collision, phi) of 32-bucket tables of every N+(u), buckets
    unbounded (Sec. 4.1, Eq. 2): hash_kind "mod32" is Algorithm 1's x mod 32,
    "mult32" the top 5 bits of x * 2654435761 mod 2^32 (multiplicative
    hashing by 2^32 / golden ratio). phi = sum_u coll(u) * maxload(u), coll(u)
    the collective out-degree sum_{v in N+(u)} d+(v)."""
    dp = np.asarray(d.dag_ptr, dtype=np.int64)
    dc = np.asarray(d.dag_col, dtype=np.int64)
    dplus = np.diff(dp)
    mx, phi = 0, 0
    for u in range(d.n):
        nu = dc[dp[u]:dp[u + 1]]
        if nu.size == 0:
            continue
        if hash_kind == "mod32":
            b = nu % 32
        elif hash_kind == "mult32":
            b = ((nu * 2654435761) % (1 << 32)) >> 27
        else:
            raise ValueError(hash_kind)
        load = int(np.bincount(b, minlength=32).max())
        mx = max(mx, load)
        phi += int(dplus[nu].sum()) * load
    return mx, phi
