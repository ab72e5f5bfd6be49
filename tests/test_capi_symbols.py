"""The C-ABI library builds for sm_103a and exports every entry point that
include/bdl.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bdl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bdl_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_06188_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_batch_operations():
    names = declared_functions()
    for n in ("bdl_create", "bdl_insert", "bdl_erase", "bdl_knn", "bdl_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2112_06188_gb300 import capi
    assert sorted(capi.SYMBOLS) == declared_functions()


def test_status_strings_without_gpu(lib):
    lib.bdl_status_string.restype = ctypes.c_char_p
    assert lib.bdl_status_string(0) == b"ok"
    assert lib.bdl_status_string(1) == b"invalid argument"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    lib.bdl_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    # dim out of range is checked before touching the device
    assert lib.bdl_create(0, None, None, ctypes.c_int64(0), None, None, ctypes.byref(out)) == 1
    assert lib.bdl_create(17, None, None, ctypes.c_int64(0), None, None, ctypes.byref(out)) == 1
    assert out.value is None
    lib.bdl_destroy.restype = ctypes.c_int
    assert lib.bdl_destroy(None) == 0


def test_new_entry_points_reject_bad_arguments_without_gpu(lib):
    """The batched, plan and server entry points validate their arguments on the
    host before any device work (so this runs without a GPU)."""
    from paper_2112_06188_gb300 import capi
    capi.load()
    P = ctypes.c_void_p
    # empty batches are no-ops
    assert capi.bdl_insert_batch([], [], [], [], None) == capi.BDL_OK
    assert capi.bdl_erase_batch([], [], [], None)[0] == capi.BDL_OK
    assert capi.bdl_knn_batch([], [], [], 5, [], [], None) == capi.BDL_OK
    # a NULL forest in a batch
    assert capi.bdl_insert_batch([None], [None], [0], [None], None) == capi.BDL_EINVAL
    assert capi.bdl_knn_batch([None], [None], [0], 5, [None], [None], None) == capi.BDL_EINVAL
    # plans need at least one forest
    st, h = capi.bdl_knn_plan_create([], [], [], 5, [], [], None)
    assert st == capi.BDL_EINVAL and h is None
    assert capi.bdl_knn_plan_launch(None, None) == capi.BDL_EINVAL
    assert capi.bdl_knn_plan_destroy(None) == capi.BDL_OK
    # servers
    st, h = capi.bdl_server_create(None, None)
    assert st == capi.BDL_EINVAL and h is None
    req = capi.BdlRequest()
    assert capi.bdl_server_submit(None, req)[0] == capi.BDL_EINVAL
    assert capi.bdl_server_destroy(None) == capi.BDL_OK
    cfg = capi.bdl_server_default_config()
    assert cfg.max_inflight == 64 and cfg.serial == 0 and cfg.staging_budget_bytes == 1 << 30
    # the splitting rule is part of the configuration and is checked
    c = capi.bdl_default_config()
    assert c.split_rule == capi.BDL_SPLIT_OBJECT
    c.split_rule = 7
    out = P()
    assert lib.bdl_create(3, ctypes.byref(c), None, ctypes.c_int64(0), None, None, ctypes.byref(out)) == 1
    assert "split_rule" in capi.last_error()
