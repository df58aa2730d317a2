"""The C ABI library builds, loads and exports every symbol that
include/bkd.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1512_02831_gb300 as bkd

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include",
                      "bkd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bkd_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("bkd_build", "bkd_build_with", "bkd_query", "bkd_set_option",
              "bkd_get_stat", "bkd_free", "bkd_last_error",
              "bkd_tree_shape", "bkd_export_tree"):
        assert f in names


def test_library_exports_every_declared_symbol():
    lib = bkd.load()
    assert os.path.dirname(bkd.library_path()).endswith(
        os.path.join("paper_1512_02831_gb300", "_build"))
    for name in declared_functions():
        assert hasattr(lib, name), f"libbkd.so lacks {name}"
    # exported with C linkage (no C++ mangling)
    raw = ctypes.CDLL(bkd.library_path())
    for name in declared_functions():
        ctypes.cast(getattr(raw, name), ctypes.c_void_p)


def test_python_binding_names_match_the_abi():
    for name in declared_functions():
        if name == "bkd_build_with":   # folded into bkd_build(**options)
            continue
        assert hasattr(bkd, name), f"binding lacks {name}"


def test_build_rejects_bad_arguments_before_any_device_work():
    lib = bkd.load()
    out = ctypes.c_void_p()
    P = np.zeros((16, 3), np.float32)
    p = P.ctypes.data
    assert lib.bkd_build(None, 16, 3, 2, ctypes.byref(out)) == bkd.BKD_EINVAL
    assert lib.bkd_build(p, 0, 3, 0, ctypes.byref(out)) == bkd.BKD_EINVAL
    assert lib.bkd_build(p, 16, 0, 2, ctypes.byref(out)) == bkd.BKD_EINVAL
    assert lib.bkd_build(p, 16, 33, 2, ctypes.byref(out)) == bkd.BKD_EINVAL
    assert lib.bkd_build(p, 16, 3, 5, ctypes.byref(out)) == bkd.BKD_EINVAL
    assert "exceed" in bkd.bkd_last_error()
    assert lib.bkd_build(p, 16, 3, -1, ctypes.byref(out)) == bkd.BKD_EINVAL
    assert lib.bkd_build(p, 16, 3, 2, None) == bkd.BKD_EINVAL
    opts = (ctypes.c_int64 * 2)(99, 1)
    assert lib.bkd_build_with(p, 16, 3, 2, opts, 1,
                              ctypes.byref(out)) == bkd.BKD_EINVAL
    assert "unknown" in bkd.bkd_last_error()
    assert not out.value


def test_query_rejects_null_handle():
    lib = bkd.load()
    assert lib.bkd_query(None, None, 0, 1, None, None) == bkd.BKD_EINVAL
    assert lib.bkd_set_option(None, 1, 0) == bkd.BKD_EINVAL
    v = ctypes.c_double()
    assert lib.bkd_get_stat(None, 1, ctypes.byref(v)) == bkd.BKD_EINVAL
    lib.bkd_free(None)  # ignored


def test_binding_refuses_wrong_dtypes():
    with pytest.raises(TypeError):
        bkd.bkd_build(np.zeros((8, 2), np.float64), 1)


def test_serving_rejects_bad_arguments_before_any_device_work():
    lib = bkd.load()
    out = ctypes.c_void_p()
    assert lib.bkd_serve_open(None, 10, 100, ctypes.byref(out)) == \
        bkd.BKD_EINVAL
    assert "tree is NULL" in bkd.bkd_last_error()
    ticket = ctypes.c_int64()
    assert lib.bkd_serve_submit(None, None, 0, 1, None, None,
                                ctypes.byref(ticket)) == bkd.BKD_EINVAL
    pending = ctypes.c_int64()
    assert lib.bkd_serve_step(None, ctypes.byref(pending)) == bkd.BKD_EINVAL
    st = ctypes.c_int()
    assert lib.bkd_serve_status(None, 1, ctypes.byref(st)) == bkd.BKD_EINVAL
    lib.bkd_serve_close(None)  # NULL is ignored


def test_calls_are_ordered_after_the_callers_stream():
    """The binding's stream choice for a call on CUDA tensors: a stream with
    a handle of its own is passed on untouched; the legacy default stream
    (handle 0, which the library reads as its own stream) is first waited
    for on the host, so the call cannot read inputs still being written."""
    class FakeStream:
        def __init__(self, handle):
            self.cuda_stream = handle
            self.waits = 0

        def synchronize(self):
            self.waits += 1

    side = FakeStream(0x7f00dead0000)
    assert bkd._stream_for_call(side) == 0x7f00dead0000 and side.waits == 0
    default = FakeStream(0)
    assert bkd._stream_for_call(default) == 0 and default.waits == 1


def test_binding_constants_match_the_header():
    """Option and statistic numbers, status codes and limits of the binding
    are the values include/bkd.h defines (the binding passes them as plain
    integers, so a mismatch would silently set the wrong option)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    opts = {k.lower(): int(v)
            for k, v in re.findall(r"\bBKD_OPT_([A-Z_]+)\s*=\s*(\d+)", text)}
    stats = {k.lower(): int(v)
             for k, v in re.findall(r"\bBKD_STAT_([A-Z_]+)\s*=\s*(\d+)", text)}
    assert opts == bkd.OPTIONS
    assert stats == bkd.STATS
    defines = {k: int(v) for k, v in
               re.findall(r"#define\s+(BKD_[A-Z_]+)\s+\(?(-?\d+)\)?", text)}
    for name, value in defines.items():
        if hasattr(bkd, name):
            assert getattr(bkd, name) == value, name
    for name in ("BKD_OK", "BKD_EINVAL", "BKD_ENOMEM", "BKD_ECUDA",
                 "BKD_ETIMEOUT", "BKD_EUNSUPPORTED", "BKD_MAX_DIM",
                 "BKD_MAX_K", "BKD_MAX_HEIGHT", "BKD_STATIC_MAX_QUERIES",
                 "BKD_STATIC_MAX_HEIGHT"):
        assert name in defines and hasattr(bkd, name), name
    batch = dict(re.findall(r"\b(BKD_BATCH_[A-Z]+)\s*=\s*(\d+)", text))
    assert {k: int(v) for k, v in batch.items()} == {
        "BKD_BATCH_QUEUED": bkd.BKD_BATCH_QUEUED,
        "BKD_BATCH_RUNNING": bkd.BKD_BATCH_RUNNING,
        "BKD_BATCH_DONE": bkd.BKD_BATCH_DONE}
