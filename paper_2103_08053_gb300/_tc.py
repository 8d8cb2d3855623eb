"""ctypes binding of include/tc.h (argument marshalling only).

The functions keep the C names (``tc_create``, ``tc_count``, ...). Every
step of the counting path runs in libtrust.so's CUDA kernels; this module
only packs pointers and sizes. Importing it fails loudly when the library has
not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtrust.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "tc.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

lib = ctypes.CDLL(LIB_PATH)

c_int32, c_int64, c_uint64, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                                  ctypes.c_void_p, ctypes.c_size_t)

# tc_status
TC_OK = 0
TC_ERR_INVALID_ARG = 1
TC_ERR_BAD_GRAPH = 2
TC_ERR_OOM = 3
TC_ERR_BUSY = 4
TC_ERR_NOT_READY = 5
TC_ERR_TIMEOUT = 6
TC_ERR_CUDA = 7
TC_ERR_UNSUPPORTED = 8

# tc_reorder kinds
TC_REORDER_INDEGREE = 1
TC_REORDER_COLLECTIVE = 2

# tc_params.balance (Sec. 4.2)
TC_BALANCE_VC = 0
TC_BALANCE_WC = 1
TC_BALANCE_SW8 = 2
TC_BALANCE_SW16 = 3
TC_BALANCE_PC = 4


class tc_csr(ctypes.Structure):
    _fields_ = [("n", c_int64), ("nnz", c_int64), ("row_ptr", c_void_p), ("offset_bits", c_int32),
                ("col", c_void_p)]


class tc_dag(ctypes.Structure):
    _fields_ = [("n", c_int64), ("m", c_int64), ("dag_ptr", c_void_p), ("dag_col", c_void_p)]


class tc_params(ctypes.Structure):
    _fields_ = [("warp_max_out_degree", c_int32), ("warp_area_ints", c_int32), ("warp_min_buckets", c_int32),
                ("block_threads", c_int32), ("block_smem_bytes", c_int32),
                ("item_neighbors", c_int32), ("chunk", c_int32), ("warps_per_block", c_int32),
                ("shard_count", c_int32), ("shard_index", c_int32), ("validate", c_int32),
                ("record_timing", c_int32), ("hash_mode", c_int32), ("scalar_loads", c_int32),
                ("edge_centric", c_int32), ("balance", c_int32),
                ("warp_order", c_int32)]


class tc_timing(ctypes.Structure):
    _fields_ = [("calls", c_int64), ("orient_ms", ctypes.c_double), ("bin_ms", ctypes.c_double),
                ("count_ms", ctypes.c_double), ("build_cycles", c_int64), ("probe_cycles", c_int64)]


class tc_stats(ctypes.Structure):
    _fields_ = [("n", c_int64), ("m", c_int64), ("max_out_degree", c_int64), ("n_skip", c_int64),
                ("n_warp", c_int64), ("n_block", c_int64), ("wedges_plus", c_int64),
                ("wedges_plus_block", c_int64),
                ("max_collision_mod32", c_int64), ("max_collision_mult32", c_int64),
                ("phi_mod32", c_int64), ("phi_mult32", c_int64)]


_P = ctypes.POINTER
_protos = {
    "tc_default_params": (c_int32, [_P(tc_params)]),
    "tc_create": (c_int32, [_P(c_void_p), ctypes.c_int, c_size_t, _P(tc_params)]),
    "tc_destroy": (c_int32, [c_void_p]),
    "tc_set_params": (c_int32, [c_void_p, _P(tc_params)]),
    "tc_get_params": (c_int32, [c_void_p, _P(tc_params)]),
    "tc_orient": (c_int32, [c_void_p, _P(tc_csr), _P(tc_dag), c_void_p]),
    "tc_dag_free": (c_int32, [c_void_p, _P(tc_dag)]),
    "tc_count_dag": (c_int32, [c_void_p, _P(tc_dag), _P(c_uint64), c_void_p, c_void_p]),
    "tc_count": (c_int32, [c_void_p, _P(tc_csr), _P(c_uint64), c_void_p]),
    "tc_count_async": (c_int32, [c_void_p, _P(tc_csr), c_void_p, c_void_p, c_void_p]),
    "tc_reserve": (c_int32, [c_void_p, c_int64, c_int64]),
    "tc_count_host": (c_int32, [c_void_p, _P(tc_csr), _P(c_uint64), c_void_p]),
    "tc_dag_stats": (c_int32, [c_void_p, _P(tc_dag), _P(tc_stats), c_void_p]),
    "tc_count_batch": (c_int32, [c_void_p, _P(tc_csr), c_int32, _P(c_uint64), c_void_p]),
    "tc_autotune": (c_int32, [c_void_p, _P(tc_csr), c_int32, ctypes.c_char_p, _P(tc_params), c_void_p]),
    "tc_submit": (c_int32, [c_void_p, _P(tc_csr), _P(c_uint64)]),
    "tc_submit_borrowed": (c_int32, [c_void_p, _P(tc_csr), _P(c_uint64)]),
    "tc_poll": (c_int32, [c_void_p, c_uint64, _P(c_uint64)]),
    "tc_drain": (c_int32, [c_void_p]),
    "tc_read_timing": (c_int32, [c_void_p, _P(tc_timing)]),
    "tc_count_dag_noalloc": (c_int32, [_P(tc_dag), c_void_p, c_void_p, c_void_p]),
    "tc_reorder": (c_int32, [c_void_p, _P(tc_csr), c_int32, c_void_p, _P(tc_csr), c_void_p]),
    "tc_kernel_launches": (c_int32, [c_void_p, _P(c_int64)]),
    "tc_inject_oom": (c_int32, [c_void_p, c_int64]),
    "tc_status_string": (ctypes.c_char_p, [c_int32]),
    "tc_last_error": (ctypes.c_char_p, [c_void_p]),
    "tc_version": (ctypes.c_char_p, []),
}

for _name, (_res, _args) in _protos.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


def declared_functions(header: str = HEADER) -> list:
    """Names of the functions include/tc.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", text)))


def exported(name: str) -> bool:
    try:
        getattr(lib, name)
        return True
    except AttributeError:
        return False
