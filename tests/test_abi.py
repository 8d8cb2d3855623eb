"""The C-ABI library builds, loads and exports what include/tc.h declares.

No compute call is made here (these run without a GPU).
"""
import ast
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tc():
    import __graft_entry__ as ge
    ge._load_builder().build()
    from paper_2103_08053_gb300 import _tc
    return _tc


def test_every_declared_symbol_is_exported(tc):
    names = tc.declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not tc.exported(n)]
    assert not missing, missing
    for core in ("tc_orient", "tc_count", "tc_count_batch", "tc_submit", "tc_poll"):
        assert core in names


def test_status_strings(tc):
    for code in range(9):
        s = tc.tc_status_string(code).decode()
        assert s.startswith("TC_")
    assert tc.tc_status_string(99).decode() == "unknown tc_status"
    assert b"sm_103a" in tc.tc_version()


def test_default_params(tc):
    import paper_2103_08053_gb300 as T
    p = T.default_params()
    assert p["warp_min_buckets"] & (p["warp_min_buckets"] - 1) == 0
    assert p["item_neighbors"] <= p["block_threads"]
    assert p["shard_count"] == 1 and p["shard_index"] == 0
    assert p["balance"] == T.TC_BALANCE_VC == 0 and p["warp_order"] == 0
    assert (T.TC_BALANCE_WC, T.TC_BALANCE_SW8, T.TC_BALANCE_SW16, T.TC_BALANCE_PC) == (1, 2, 3, 4)


def test_params_struct_matches_header(tc):
    # the ctypes mirror of tc_params has the header's fields, in order
    import re
    hdr = open(os.path.join(ROOT, "include", "tc.h")).read()
    end = hdr.index("} tc_params;")
    body = hdr[hdr.rindex("typedef struct", 0, end):end]
    fields = re.findall(r"int32_t\s+(\w+)(?:\[\d+\])?;", body)
    assert fields == [f for f, _ in tc.tc_params._fields_]


def test_null_arguments_rejected_without_gpu(tc):
    import ctypes
    assert tc.tc_count(None, None, None, None) == tc.TC_ERR_INVALID_ARG
    assert tc.tc_destroy(None) == tc.TC_OK
    assert tc.tc_default_params(None) == tc.TC_ERR_INVALID_ARG
    assert tc.tc_inject_oom(None, 1) == tc.TC_ERR_INVALID_ARG
    assert isinstance(tc.tc_last_error(None), bytes)


def test_create_fails_cleanly_without_gpu(tc):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    h = ctypes.c_void_p()
    assert tc.tc_create(ctypes.byref(h), 0, 0, None) == tc.TC_ERR_CUDA


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2103_08053_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
            if isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", path
    for path in glob.glob(os.path.join(pkg, "csrc", "*")):
        assert "oracle" not in open(path).read().lower(), path


def test_oracle_and_cuda_share_no_sources():
    orc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "#include \"tc" not in orc and "tc_internal" not in orc
