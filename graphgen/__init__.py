"""Seeded synthetic graph generators (inputs only).

Everything here produces simple undirected graphs as a symmetric CSR
(``row_ptr`` int64[n+1], ``col`` int32[nnz], rows sorted, no self-loops, no
duplicates). None of the triangle-counting arithmetic lives here: both the CPU
oracle's tests and the GPU path's tests and bench draw their inputs from this
module, and the two sides share nothing else.

The bulk generators (R-MAT, G(n,p), random geometric graphs, edge list -> CSR)
are C in ``graphgen.c`` (compiled on first use, or by ``build()``); the small
closed-form families used as test pins are plain numpy.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib_handle = None

I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)
F64P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, OpenMP if available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", tmp]
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
            lib.gg_stream_key.restype = ctypes.c_uint64
            lib.gg_stream_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_draw.restype = ctypes.c_uint64
            lib.gg_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_u01.restype = ctypes.c_double
            lib.gg_u01.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_log.restype = ctypes.c_double
            lib.gg_log.argtypes = [ctypes.c_double]
            lib.gg_exp2.restype = ctypes.c_double
            lib.gg_exp2.argtypes = [ctypes.c_double]
            lib.gg_rmat_edges.restype = None
            lib.gg_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, I32P, I32P]
            lib.gg_er_edges.restype = ctypes.c_int64
            lib.gg_er_edges.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                        I32P, I32P]
            lib.gg_rgg_points.restype = None
            lib.gg_rgg_points.argtypes = [ctypes.c_int64, ctypes.c_uint64, F64P, F64P]
            lib.gg_rgg_csr.restype = ctypes.c_int64
            lib.gg_rgg_csr.argtypes = [ctypes.c_int64, F64P, F64P, ctypes.c_double, I64P, I32P]
            lib.gg_build_csr.restype = ctypes.c_int64
            lib.gg_build_csr.argtypes = [ctypes.c_int64, ctypes.c_int64, I32P, I32P, I64P, I32P]
            lib.gg_batch_spec.restype = None
            lib.gg_batch_spec.argtypes = [ctypes.c_uint64, ctypes.c_int64, I32P, I64P, F64P]
            lib.gg_num_threads.restype = ctypes.c_int
            lib.gg_set_threads.restype = None
            lib.gg_set_threads.argtypes = [ctypes.c_int]
            _lib_handle = lib
    return _lib_handle


def _p(a, t):
    return a.ctypes.data_as(t)


@dataclasses.dataclass
class Csr:
    """Symmetric CSR of a simple undirected graph."""

    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        """Undirected edge count (each edge is stored twice)."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def row(self, u: int) -> np.ndarray:
        return self.col[self.row_ptr[u]:self.row_ptr[u + 1]]


# ------------------------------------------------------------------ bulk (C)

def stream_key(seed: int, stream: int) -> int:
    return int(_lib().gg_stream_key(seed & (2**64 - 1), stream & (2**64 - 1)))


def csr_from_edges(n: int, src, dst, name: str = "") -> Csr:
    """Symmetrise, drop self-loops/out-of-range, deduplicate, sort rows."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    ne = int(src.shape[0])
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(2 * ne, 1), dtype=np.int32)
    nnz = _lib().gg_build_csr(n, ne, _p(src, I32P), _p(dst, I32P), _p(row_ptr, I64P), _p(col, I32P))
    if nnz < 0:
        raise MemoryError("gg_build_csr: allocation failed")
    col = col[:nnz]
    return Csr(n, row_ptr, col, name)


def rmat_edges(scale: int, n_edges: int, seed: int, stream: int = 0, a=0.57, b=0.19, c=0.19,
               n_keep: int | None = None):
    src = np.empty(n_edges, dtype=np.int32)
    dst = np.empty(n_edges, dtype=np.int32)
    key = stream_key(seed, stream)
    nk = (1 << scale) if n_keep is None else n_keep
    _lib().gg_rmat_edges(scale, n_edges, a, b, c, key, nk, _p(src, I32P), _p(dst, I32P))
    return src, dst


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, a=0.57, b=0.19, c=0.19, n: int | None = None,
         stream: int = 0) -> Csr:
    """R-MAT graph: edge_factor * 2^scale generated edges, then symmetrised and
    deduplicated; n = 2^scale unless given (ids >= n are redrawn)."""
    nv = (1 << scale) if n is None else n
    ne = edge_factor * (1 << scale) if n is None else edge_factor * nv
    src, dst = rmat_edges(scale, ne, seed, stream, a, b, c, nv)
    g = csr_from_edges(nv, src, dst, name=f"rmat-s{scale}-ef{edge_factor}-seed{seed}")
    del src, dst
    return g


def erdos_renyi(n: int, p: float, seed: int, stream: int = 0) -> Csr:
    """G(n, p) by geometric skipping (Batagelj & Brandes 2005)."""
    key = stream_key(seed, stream)
    lib = _lib()
    cap = int(p * n * (n - 1) / 2 * 1.2 + 64)
    while True:
        src = np.empty(cap, dtype=np.int32)
        dst = np.empty(cap, dtype=np.int32)
        m = lib.gg_er_edges(n, p, key, cap, _p(src, I32P), _p(dst, I32P))
        if m <= cap:
            break
        cap = int(m) + 16
    return csr_from_edges(n, src[:m], dst[:m], name=f"er-n{n}-p{p:.4g}-seed{seed}")


def rgg_radius(n: int, mean_degree: float) -> float:
    """r with n * pi * r^2 = mean degree (ignoring the boundary)."""
    return math.sqrt(mean_degree / (math.pi * n))


def rgg(n: int, mean_degree: float = 64.0, seed: int = 2, r: float | None = None) -> Csr:
    """Random geometric graph: n uniform points in [0,1)^2 (ids in generation
    order), edge iff Euclidean distance < r, no wrap-around."""
    rr = rgg_radius(n, mean_degree) if r is None else r
    lib = _lib()
    x = np.empty(n, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    lib.gg_rgg_points(n, stream_key(seed, 0), _p(x, F64P), _p(y, F64P))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    nnz = lib.gg_rgg_csr(n, _p(x, F64P), _p(y, F64P), rr, _p(row_ptr, I64P), None)
    if nnz < 0:
        raise MemoryError("gg_rgg_csr: allocation failed")
    col = np.empty(max(nnz, 1), dtype=np.int32)
    lib.gg_rgg_csr(n, _p(x, F64P), _p(y, F64P), rr, _p(row_ptr, I64P), _p(col, I32P))
    return Csr(n, row_ptr, col[:nnz], name=f"rgg-n{n}-r{rr:.6g}-seed{seed}")


# --------------------------------------------------- batched workload graphs

BATCH_EDGE_STREAM = 1 << 40


def batch_spec(seed: int, idx: int):
    """(kind, n, mean_degree) of graph idx: kind 0 = G(n,p), 1 = R-MAT."""
    k = ctypes.c_int32()
    n = ctypes.c_int64()
    d = ctypes.c_double()
    _lib().gg_batch_spec(seed, idx, ctypes.byref(k), ctypes.byref(n), ctypes.byref(d))
    return int(k.value), int(n.value), float(d.value)


def batch_graph(seed: int, idx: int) -> Csr:
    """Graph idx of the batched workload: G(n,p) with p = d/(n-1), or R-MAT
    (0.57, 0.19, 0.19, 0.05) at scale ceil(log2 n) with n*d/2 edges whose
    endpoints >= n are redrawn."""
    kind, n, d = batch_spec(seed, idx)
    stream = BATCH_EDGE_STREAM + idx
    if kind == 0:
        g = erdos_renyi(n, d / (n - 1), seed, stream)
    else:
        scale = max(1, (n - 1).bit_length())
        ne = int(round(n * d / 2.0))
        src, dst = rmat_edges(scale, ne, seed, stream, n_keep=n)
        g = csr_from_edges(n, src, dst)
    g.name = f"batch-seed{seed}-{idx}-{'er' if kind == 0 else 'rmat'}-n{n}"
    return g


def batch(seed: int, k: int, threads: int = 0) -> list:
    """Graphs 0..k-1 of the batched workload, generated by `threads` host
    threads (default: all cores), each running its C calls single-threaded."""
    import concurrent.futures as cf
    threads = threads or os.cpu_count() or 1
    if threads == 1:
        return [batch_graph(seed, i) for i in range(k)]
    lib = _lib()

    def one(i):
        lib.gg_set_threads(1)
        return batch_graph(seed, i)

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, range(k)))


# --------------------------------------------- small closed-form families

def from_edge_list(n: int, edges, name: str = "") -> Csr:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), name)


def empty(n: int) -> Csr:
    return Csr(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), f"empty-{n}")


def complete(n: int) -> Csr:
    """K_n."""
    i, j = np.triu_indices(n, 1)
    return csr_from_edges(n, i.astype(np.int32), j.astype(np.int32), f"K{n}")


def cycle(n: int) -> Csr:
    """C_n (n >= 3)."""
    i = np.arange(n)
    return csr_from_edges(n, i.astype(np.int32), ((i + 1) % n).astype(np.int32), f"C{n}")


def wheel(n: int) -> Csr:
    """W_n: hub 0 joined to every vertex of the cycle 1..n."""
    i = np.arange(n)
    rim_s, rim_d = 1 + i, 1 + (i + 1) % n
    src = np.concatenate([rim_s, np.zeros(n, dtype=np.int64)])
    dst = np.concatenate([rim_d, 1 + i])
    return csr_from_edges(n + 1, src.astype(np.int32), dst.astype(np.int32), f"W{n}")


def friendship(k: int) -> Csr:
    """F_k: k triangles sharing the centre 0."""
    e = []
    for t in range(k):
        a, b = 1 + 2 * t, 2 + 2 * t
        e += [(0, a), (0, b), (a, b)]
    return from_edge_list(2 * k + 1, e, f"F{k}")


def complete_bipartite(a: int, b: int) -> Csr:
    i, j = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return csr_from_edges(a + b, i.ravel().astype(np.int32), j.ravel().astype(np.int32), f"K{a},{b}")


def star(n: int) -> Csr:
    """Hub 0 with n leaves."""
    return csr_from_edges(n + 1, np.zeros(n, dtype=np.int32), np.arange(1, n + 1, dtype=np.int32), f"S{n}")


def grid2d(a: int, b: int) -> Csr:
    idx = np.arange(a * b).reshape(a, b)
    src = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    dst = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return csr_from_edges(a * b, src.astype(np.int32), dst.astype(np.int32), f"grid{a}x{b}")


def torus3d(s: int) -> Csr:
    """s^3 periodic 3D grid (every vertex has 6 neighbours for s >= 3)."""
    idx = np.arange(s ** 3, dtype=np.int64).reshape(s, s, s)
    srcs, dsts = [], []
    for ax in range(3):
        srcs.append(idx.ravel())
        dsts.append(np.roll(idx, -1, axis=ax).ravel())
    return csr_from_edges(s ** 3, np.concatenate(srcs).astype(np.int32),
                          np.concatenate(dsts).astype(np.int32), f"torus{s}^3")


def disjoint_union(gs) -> Csr:
    offs = np.cumsum([0] + [g.n for g in gs])
    rp = [np.zeros(1, dtype=np.int64)]
    cols = []
    base = 0
    for g, o in zip(gs, offs[:-1]):
        rp.append(g.row_ptr[1:] + base)
        cols.append(g.col.astype(np.int64) + o)
        base += g.nnz
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, dtype=np.int32)
    return Csr(int(offs[-1]), np.concatenate(rp), col, "union")


def relabel(g: Csr, perm: np.ndarray) -> Csr:
    """Graph with vertex v renamed perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return csr_from_edges(g.n, perm[src].astype(np.int32), perm[g.col].astype(np.int32), g.name + "-relabel")


def shuffle_rows(g: Csr, seed: int) -> Csr:
    """Same graph with every row's neighbour order permuted (rows unsorted)."""
    rng = np.random.default_rng(seed)
    col = g.col.copy()
    for u in range(g.n):
        b, e = g.row_ptr[u], g.row_ptr[u + 1]
        if e - b > 1:
            col[b:e] = rng.permutation(col[b:e])
    return Csr(g.n, g.row_ptr.copy(), col, g.name + "-shuffled")


def random_small(n: int, p: float, seed: int) -> Csr:
    """Small G(n,p) drawn with numpy (test inputs)."""
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(n, 1)
    keep = rng.random(i.shape[0]) < p
    return csr_from_edges(n, i[keep].astype(np.int32), j[keep].astype(np.int32), f"gnp{n}-{p}-{seed}")


# ------------------------------------------------------- workload recipes

def workload(name: str) -> Csr:
    """The named synthetic workloads:
    rmat16 -- R-MAT scale 16, edge factor 16, (0.57, 0.19, 0.19, 0.05), seed 1;
    rgg22  -- 2^22 uniform points in the unit square, r for mean degree 64, seed 2;
    rmat26 -- R-MAT scale 26, edge factor 16, seed 3 (int64 offsets needed on device).
    """
    if name == "rmat16":
        return rmat(16, 16, seed=1)
    if name == "rgg22":
        return rgg(1 << 22, 64.0, seed=2)
    if name == "rmat26":
        return rmat(26, 16, seed=3)
    if name.startswith("rmat") and name[4:].isdigit():
        return rmat(int(name[4:]), 16, seed=1)
    if name.startswith("rgg") and name[3:].isdigit():
        return rgg(1 << int(name[3:]), 64.0, seed=2)
    raise KeyError(name)
