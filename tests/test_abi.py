"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/cafs.h declares, and rejects bad arguments before any
device work (these paths never touch CUDA)."""

import ctypes
import os
import re

import pytest

from paper_2605_25040_gb300 import build as B
from paper_2605_25040_gb300 import cafs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cafs_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cafs.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "cafs_sort" in declared and "cafs_estimate_k" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(cafs.SIGNATURES), "binding misses a declared function"


def test_argument_errors_are_synchronous(lib):
    buf = (ctypes.c_int64 * 16)()
    p = ctypes.addressof(buf)
    # unsupported dtype
    assert lib.cafs_sort(p, 4, 7, p + 64, None) == 2
    # n == 0 is a no-op even with NULL pointers
    assert lib.cafs_sort(None, 0, cafs.INT64, None, None) == 0
    # n > 2^32 - 1
    assert lib.cafs_sort(p, 1 << 32, cafs.INT64, p + 64, None) == 3
    # NULL keys / out
    assert lib.cafs_sort(None, 4, cafs.INT64, p, None) == 1
    assert lib.cafs_sort(p, 4, cafs.INT64, None, None) == 1
    # misaligned for the element type
    assert lib.cafs_sort(p + 4, 4, cafs.INT64, p + 64, None) == 1
    # partial overlap of keys and out
    assert lib.cafs_sort(p, 8, cafs.INT64, p + 8, None) == 4
    est = cafs.Estimate()
    assert lib.cafs_estimate_k(p, 4, 9, ctypes.byref(est), None) == 2
    assert lib.cafs_estimate_k(p, 4, cafs.INT64, None, None) == 1


def test_argsort_argument_errors_are_synchronous(lib):
    buf = (ctypes.c_int64 * 64)()
    p = ctypes.addressof(buf)
    # n == 0: a no-op with NULL pointers
    assert lib.cafs_argsort(None, 0, cafs.INT64, None, None, None, None) == 0
    assert lib.cafs_argsort(p, 4, 6, p + 64, p + 128, None, None) == 2
    assert lib.cafs_argsort(p, 1 << 32, cafs.INT64, p + 64, p + 128, None, None) == 3
    # NULL out or perm, misaligned perm
    assert lib.cafs_argsort(p, 4, cafs.INT64, None, p + 128, None, None) == 1
    assert lib.cafs_argsort(p, 4, cafs.INT64, p + 64, None, None, None) == 1
    assert lib.cafs_argsort(p, 4, cafs.INT64, p + 64, p + 130, None, None) == 1
    # keys, out and perm must be pairwise disjoint (keys == out too)
    assert lib.cafs_argsort(p, 4, cafs.INT64, p, p + 128, None, None) == 4
    assert lib.cafs_argsort(p, 4, cafs.INT64, p + 64, p + 16, None, None) == 4
    assert lib.cafs_argsort(p, 4, cafs.INT64, p + 64, p + 80, None, None) == 4
    assert lib.cafs_argsort(p, 4, cafs.INT32, p + 64, p + 72, None, None) == 4


def test_key_types(lib):
    buf = (ctypes.c_int64 * 64)()
    p = ctypes.addressof(buf)
    # 8-byte key types need 8-byte alignment, 4-byte ones 4-byte
    assert lib.cafs_sort(p + 4, 4, cafs.UINT64, p + 64, None) == 1
    assert lib.cafs_sort(p + 4, 4, cafs.FLOAT64, p + 64, None) == 1
    assert lib.cafs_sort(p, 8, cafs.FLOAT32, p + 4, None) == 4
    # the allocation-free entry point takes int32/int64 only; the batched form
    # checks every column's type (6 is no type)
    for t in (cafs.UINT32, cafs.UINT64, cafs.FLOAT32, cafs.FLOAT64):
        assert lib.cafs_sort_noalloc(p, 4, t, p + 64, None) == 2
    cols = (cafs.Column * 1)()
    cols[0].keys, cols[0].out, cols[0].n, cols[0].dtype = p, p + 256, 8, 6
    assert lib.cafs_sort_batch(cols, 1, None, None) == 2
    cols[0].dtype = cafs.FLOAT64
    cols[0].keys = p + 4                       # misaligned 8-byte keys
    assert lib.cafs_sort_batch(cols, 1, None, None) == 1
    assert cafs.KEY_TYPES["float64"] == (cafs.FLOAT64, 8)


def test_names(lib):
    assert lib.cafs_status_string(0) == b"ok"
    assert lib.cafs_path_string(4) == b"main"
    assert lib.cafs_path_string(8) == b"tiny_miss_main_overflow_radix"
    for code, name in cafs.PATHS.items():
        assert lib.cafs_path_string(code).decode() == name


def test_batch_argument_errors_are_synchronous(lib):
    buf = (ctypes.c_int64 * 64)()
    p = ctypes.addressof(buf)
    cols = (cafs.Column * 2)()
    cols[0].keys, cols[0].out, cols[0].n, cols[0].dtype = p, p + 256, 8, cafs.INT64
    cols[1].keys, cols[1].out, cols[1].n, cols[1].dtype = p + 128, p + 128, 8, 6
    # an unsupported dtype in any column rejects the whole batch before any work
    assert lib.cafs_sort_batch(cols, 2, None, None) == 2
    cols[1].dtype = cafs.INT64
    cols[1].reserved = 1
    assert lib.cafs_sort_batch(cols, 2, None, None) == 1
    cols[1].reserved = 0
    cols[1].out = p + 136          # partial overlap inside one column
    assert lib.cafs_sort_batch(cols, 2, None, None) == 4
    cols[1].out = p + 128
    # bad knobs
    for bad in ({"local_slots_max": 300}, {"local_slots_max": 16384}, {"replicas_max": 3},
                {"emit_tile_vec": 1000}, {"emit_tile_vec": 16384}, {"grid_min_n": 100},
                {"cta_table_slots": 1000}, {"cta_table_slots": 32}):
        t = cafs.BatchTuning.from_dict(bad)
        assert lib.cafs_sort_batch_tuned(cols, 2, ctypes.byref(t), None, None) == 1, bad
        h = ctypes.c_void_p()
        assert lib.cafs_batch_plan_create(cols, 2, ctypes.byref(t), ctypes.byref(h)) == 1, bad
        assert not h.value
    assert lib.cafs_sort_batch(None, 3, None, None) == 1
    assert lib.cafs_batch_plan_create(cols, 2, None, None) == 1


def test_batch_tuning_defaults(lib):
    t = cafs.BatchTuning()
    assert lib.cafs_batch_tuning_default(ctypes.byref(t)) == 0
    d = t.as_dict()
    assert d == {"grid_min_n": 0, "defer_min_n": 0, "cta_table_slots": 0, "local_slots_max": 8192,
                 "replicas_max": 32, "emit_tile_vec": 4096, "ctas": 0}
    with pytest.raises(KeyError):
        cafs.BatchTuning.from_dict({"block": 3})


def test_server_config_errors_are_synchronous(lib):
    c = cafs.ServerConfig()
    assert lib.cafs_server_config_default(ctypes.byref(c)) == 0
    assert c.max_batch_columns == 1024 and c.max_inflight == 3 and c.max_request_keys == 1 << 22
    assert c.tuning.cta_table_slots == 1 << 18 and c.tuning.grid_min_n == 0
    h = ctypes.c_void_p()
    bad = cafs.ServerConfig.from_buffer_copy(c)
    bad.max_batch_columns = 0
    assert lib.cafs_server_create(1 << 30, ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = cafs.ServerConfig.from_buffer_copy(c)
    bad.reserved = 1
    assert lib.cafs_server_create(1 << 30, ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = cafs.ServerConfig.from_buffer_copy(c)
    bad.tuning.replicas_max = 5
    assert lib.cafs_server_create(1 << 30, ctypes.byref(bad), ctypes.byref(h)) == 1
    assert not h.value
    req = (cafs.Request * 2)()
    arr = (ctypes.c_double * 2)(0.0, -1.0)
    lat = (ctypes.c_double * 2)()
    assert lib.cafs_serial_run_trace(req, 2, arr, lat, None, None, None) == 1   # negative arrival


def test_autotune_argument_errors(lib):
    cols = (cafs.Column * 1)()
    ms = (ctypes.c_double * 2)()
    best = ctypes.c_size_t()
    cand = (cafs.BatchTuning * 2)()
    assert lib.cafs_batch_autotune(cols, 0, cand, 0, 1, ms, ctypes.byref(best), None) == 1
    assert lib.cafs_batch_autotune(cols, 0, cand, 2, 0, ms, ctypes.byref(best), None) == 1
    cand[1].replicas_max = 3
    assert lib.cafs_batch_autotune(cols, 0, cand, 2, 1, ms, ctypes.byref(best), None) == 1


def test_workload_signature():
    torch = pytest.importorskip("torch")
    from paper_2605_25040_gb300 import autotune
    keys = [torch.zeros(1000, dtype=torch.int64), torch.zeros(70000, dtype=torch.int32)]
    assert autotune.workload_signature(keys) == "cols=2:i32=1:log2n=[9,16]:log2sum=16"


def test_binding_key_type_names():
    import numpy as np
    import torch
    assert cafs._dtype_code(np.uint32) == cafs.UINT32 and cafs._dtype_code(np.float64) == cafs.FLOAT64
    assert cafs._dtype_code(torch.float32) == cafs.FLOAT32 and cafs._dtype_code(torch.int64) == cafs.INT64
    with pytest.raises(TypeError):
        cafs._dtype_code(np.int16)
    t64 = torch.zeros(4, dtype=torch.int64)
    assert cafs._key_code(t64, "uint64") == cafs.UINT64 and cafs._key_code(t64, None) == cafs.INT64
    with pytest.raises(ValueError):
        cafs._key_code(t64, "float32")            # 4-byte type read from 8-byte elements
    with pytest.raises(KeyError):
        cafs._key_code(t64, "int8")
