"""TRUST-style exact triangle counting on one GB300 (sm_103a).

``_tc`` is the ctypes binding of include/tc.h (same function names);
``Context`` wraps it for torch device tensors and numpy host arrays. All
counting work runs in libtrust.so's CUDA kernels; PyTorch only provides
device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _tc
from ._tc import (TC_BALANCE_PC, TC_BALANCE_SW8, TC_BALANCE_SW16, TC_BALANCE_VC, TC_BALANCE_WC,
                  TC_REORDER_COLLECTIVE, TC_REORDER_INDEGREE, TC_ERR_BAD_GRAPH, TC_ERR_BUSY, TC_ERR_CUDA, TC_ERR_INVALID_ARG, TC_ERR_NOT_READY, TC_ERR_OOM,
                  TC_ERR_TIMEOUT, TC_ERR_UNSUPPORTED, TC_OK, tc_csr, tc_dag, tc_params, tc_stats, tc_timing)

__all__ = ["Context", "TcError", "Dag", "default_params", "tc_csr", "tc_dag", "tc_params", "tc_stats"]


class TcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_tc.tc_status_string(status).decode()}: {msg}")
        self.status = status


def default_params() -> dict:
    p = tc_params()
    _tc.tc_default_params(ctypes.byref(p))
    return {f: getattr(p, f) for f, _ in tc_params._fields_ if f != "reserved"}


def _params_struct(params: dict | None):
    if params is None:
        return None
    p = tc_params()
    for k, v in params.items():
        setattr(p, k, int(v))
    return p


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _offset_bits(row_ptr) -> int:
    dt = str(row_ptr.dtype)
    if dt.endswith("int64"):
        return 64
    if dt.endswith("int32"):
        return 32
    raise TypeError(f"row_ptr must be int32 or int64, got {dt}")


def make_csr(n: int, row_ptr, col) -> tc_csr:
    """tc_csr over two arrays (torch device tensors or numpy host arrays)."""
    if str(col.dtype)[-5:] != "int32":
        raise TypeError("col must be int32")
    return tc_csr(int(n), int(col.shape[0]), _ptr(row_ptr), _offset_bits(row_ptr), _ptr(col))


class _DevArray:
    """Exposes a raw device pointer to torch via __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": (int(n),), "typestr": typestr,
                                         "strides": None, "version": 3}


class Dag:
    """A context-owned oriented graph (tc_orient result)."""

    def __init__(self, ctx: "Context", d: tc_dag):
        self.ctx = ctx
        self.raw = d

    @property
    def n(self) -> int:
        return int(self.raw.n)

    @property
    def m(self) -> int:
        return int(self.raw.m)

    def tensors(self):
        """(dag_ptr, dag_col) as torch int32 device tensors sharing the memory."""
        import torch
        dev = torch.device("cuda", self.ctx.device)
        dp = torch.as_tensor(_DevArray(self.raw.dag_ptr, self.n + 1, "<i4"), device=dev)
        dc = torch.as_tensor(_DevArray(self.raw.dag_col, max(self.m, 0), "<i4"), device=dev) if self.m else \
            torch.zeros(0, dtype=torch.int32, device=dev)
        return dp, dc

    def free(self):
        if self.raw.dag_ptr:
            self.ctx._check(_tc.tc_dag_free(self.ctx.handle, ctypes.byref(self.raw)))


class Context:
    """One tc_ctx on one device."""

    def __init__(self, device: int = 0, mem_budget: int = 0, params: dict | None = None):
        self.device = device
        h = ctypes.c_void_p()
        p = _params_struct(params)
        st = _tc.tc_create(ctypes.byref(h), device, mem_budget, ctypes.byref(p) if p is not None else None)
        if st != TC_OK:
            raise TcError(st, "tc_create: " + _tc.tc_last_error(None).decode(errors="replace"))
        self.handle = h

    def close(self):
        if self.handle:
            _tc.tc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st: int):
        if st != TC_OK:
            raise TcError(st, _tc.tc_last_error(self.handle).decode(errors="replace"))

    # params
    def set_params(self, params: dict):
        p = _params_struct(params)
        self._check(_tc.tc_set_params(self.handle, ctypes.byref(p)))

    def get_params(self) -> dict:
        p = tc_params()
        self._check(_tc.tc_get_params(self.handle, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in tc_params._fields_ if f != "reserved"}

    # hot path
    def count(self, n: int, row_ptr, col, stream=None) -> int:
        g = make_csr(n, row_ptr, col)
        out = ctypes.c_uint64()
        self._check(_tc.tc_count(self.handle, ctypes.byref(g), ctypes.byref(out), _stream_handle(stream)))
        return int(out.value)

    def count_async(self, n: int, row_ptr, col, count_out, err_out=None, stream=None):
        g = make_csr(n, row_ptr, col)
        self._check(_tc.tc_count_async(self.handle, ctypes.byref(g), ctypes.c_void_p(_ptr(count_out)),
                                       ctypes.c_void_p(_ptr(err_out)), _stream_handle(stream)))

    def reserve(self, n: int, nnz: int):
        self._check(_tc.tc_reserve(self.handle, int(n), int(nnz)))

    def count_host(self, n: int, row_ptr: np.ndarray, col: np.ndarray, stream=None) -> int:
        g = make_csr(n, row_ptr, col)
        out = ctypes.c_uint64()
        self._check(_tc.tc_count_host(self.handle, ctypes.byref(g), ctypes.byref(out), _stream_handle(stream)))
        return int(out.value)

    def orient(self, n: int, row_ptr, col, stream=None) -> Dag:
        g = make_csr(n, row_ptr, col)
        d = tc_dag()
        self._check(_tc.tc_orient(self.handle, ctypes.byref(g), ctypes.byref(d), _stream_handle(stream)))
        return Dag(self, d)

    def count_dag(self, dag, per_vertex=None, stream=None) -> int:
        d = dag.raw if isinstance(dag, Dag) else dag
        out = ctypes.c_uint64()
        self._check(_tc.tc_count_dag(self.handle, ctypes.byref(d), ctypes.byref(out),
                                     ctypes.c_void_p(_ptr(per_vertex)), _stream_handle(stream)))
        return int(out.value)

    def dag_stats(self, dag, stream=None) -> dict:
        d = dag.raw if isinstance(dag, Dag) else dag
        s = tc_stats()
        self._check(_tc.tc_dag_stats(self.handle, ctypes.byref(d), ctypes.byref(s), _stream_handle(stream)))
        return {f: int(getattr(s, f)) for f, _ in tc_stats._fields_}

    def reorder(self, n: int, row_ptr, col, kind: int, relabel: bool = True, stream=None):
        """tc_reorder (Sec. 4.1): new_id (device int32[n]) and, with relabel,
        the relabelled CSR (row_ptr, col) as new device tensors."""
        import torch
        dev = col.device
        new_id = torch.empty(max(int(n), 1), dtype=torch.int32, device=dev)
        g = make_csr(n, row_ptr, col)
        out = None
        if relabel:
            rp2 = torch.empty_like(row_ptr)
            col2 = torch.empty_like(col)
            out = make_csr(n, rp2, col2)
        self._check(_tc.tc_reorder(self.handle, ctypes.byref(g), int(kind), ctypes.c_void_p(_ptr(new_id)),
                                   ctypes.byref(out) if out is not None else None, _stream_handle(stream)))
        new_id = new_id[:int(n)]
        return (new_id, rp2, col2) if relabel else new_id

    # diagnostics
    def read_timing(self) -> dict:
        t = tc_timing()
        self._check(_tc.tc_read_timing(self.handle, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in tc_timing._fields_}

    def kernel_launches(self) -> int:
        v = ctypes.c_int64()
        self._check(_tc.tc_kernel_launches(self.handle, ctypes.byref(v)))
        return int(v.value)

    def inject_oom(self, nth: int):
        """tc_inject_oom: the nth device allocation from now fails (host-side)."""
        self._check(_tc.tc_inject_oom(self.handle, int(nth)))

    # batch
    def count_batch(self, graphs, stream=None) -> list:
        """graphs: sequence of (n, row_ptr, col) device arrays."""
        k = len(graphs)
        arr = (tc_csr * max(k, 1))()
        for i, (n, rp, col) in enumerate(graphs):
            arr[i] = make_csr(n, rp, col)
        out = (ctypes.c_uint64 * max(k, 1))()
        self._check(_tc.tc_count_batch(self.handle, arr, k, out, _stream_handle(stream)))
        return [int(out[i]) for i in range(k)]

    def autotune(self, graphs, cache_path: str | None = None, stream=None) -> dict:
        """Tune the worker/table parameters on `graphs` ((n, row_ptr, col)
        device arrays); keeps the best on this context and returns them."""
        k = len(graphs)
        arr = (tc_csr * max(k, 1))()
        for i, (n, rp, col) in enumerate(graphs):
            arr[i] = make_csr(n, rp, col)
        p = tc_params()
        self._check(_tc.tc_autotune(self.handle, arr, k, cache_path.encode() if cache_path else None,
                                    ctypes.byref(p), _stream_handle(stream)))
        return {f: getattr(p, f) for f, _ in tc_params._fields_ if f != "reserved"}

    # serving
    def submit(self, n: int, row_ptr: np.ndarray, col: np.ndarray) -> int:
        g = make_csr(n, row_ptr, col)
        t = ctypes.c_uint64()
        self._check(_tc.tc_submit(self.handle, ctypes.byref(g), ctypes.byref(t)))
        return int(t.value)

    def submit_borrowed(self, n: int, row_ptr, col) -> int:
        """Zero-copy submission: row_ptr / col (host arrays, ideally pinned) must
        stay alive and unchanged until poll() returns the count."""
        g = make_csr(n, row_ptr, col)
        t = ctypes.c_uint64()
        self._check(_tc.tc_submit_borrowed(self.handle, ctypes.byref(g), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int):
        """The count, or None while the request is not finished."""
        out = ctypes.c_uint64()
        st = _tc.tc_poll(self.handle, ticket, ctypes.byref(out))
        if st == TC_ERR_NOT_READY:
            return None
        self._check(st)
        return int(out.value)

    def drain(self):
        self._check(_tc.tc_drain(self.handle))
