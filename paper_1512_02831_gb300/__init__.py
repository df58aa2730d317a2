"""GB300 buffer k-d tree: exact k-nearest-neighbour search on one GPU.

Thin Python binding of the C ABI declared in ``include/bkd.h``.  It only
marshals arguments: every step of the search (FindLeafBatch, buffer
insertion, ProcessAllBuffers, the chunk streamer, the binary64 re-check) runs
in the CUDA library ``_build/libbkd.so``.  There is no CPU path: if the
library cannot be built or loaded, every call raises.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); float32
row-major points / queries, int64 / float32 outputs.

    tree = bkd_build(P, height=8)
    idx, dist = bkd_query(tree, Q, k=10)
    bkd_free(tree)
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _build_lib

BKD_OK = 0
BKD_EINVAL = -1
BKD_ENOMEM = -2
BKD_ECUDA = -3
BKD_ETIMEOUT = -4
BKD_EUNSUPPORTED = -5
BKD_MAX_DIM = 32
BKD_MAX_K = 63
BKD_MAX_HEIGHT = 24
BKD_STATIC_MAX_QUERIES = 4096
BKD_STATIC_MAX_HEIGHT = 16
BKD_BATCH_QUEUED, BKD_BATCH_RUNNING, BKD_BATCH_DONE = 0, 1, 2

OPTIONS = {"stream": 1, "device_mem_cap": 2, "chunks": 3, "max_active": 4,
           "tail_queries": 5, "precision": 6, "point_chunks": 7,
           "screen_tile": 8, "round_batch": 9, "screen_ctas": 10,
           "screen_kernel": 11, "rescue_rounds": 12, "defer_queries": 13}
STATS = {"rounds": 1, "leaf_visits": 2, "pairs": 3, "resorted": 4,
         "fallback": 5, "leaf_kernel_ms": 6, "chunk_bytes": 7, "copy_ms": 8,
         "leaf_launches": 9, "kernel_launches": 10, "tail_queries": 11,
         "tail_visits": 12, "tail_pairs": 13, "tail_ms": 14,
         "screen_kept": 15, "screen_pairs": 16, "screen_ms": 17,
         "screen_items": 18, "screen_visits": 19, "find_ms": 20,
         "bucket_ms": 21, "exact_ms": 22, "chunk_visits": 23,
         "screen_bytes": 24, "screen_queued": 25, "screen_overflow": 26,
         "leaf_bytes": 27, "host_syncs": 28, "fallback_points": 29,
         "mapped_bytes": 30}

_lock = threading.Lock()
_lib = None


class BkdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bkd error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build_lib.LIB


def load():
    """Builds (if needed) and loads libbkd.so; raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(_build_lib.build())
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.bkd_build.argtypes = [vp, i64, i32, i32, ctypes.POINTER(vp)]
        lib.bkd_build_with.argtypes = [vp, i64, i32, i32, vp, i32,
                                       ctypes.POINTER(vp)]
        lib.bkd_query.argtypes = [vp, vp, i64, i32, vp, vp]
        lib.bkd_query_static.argtypes = [vp, vp, i64, i32, vp, vp]
        lib.bkd_set_option.argtypes = [vp, i32, i64]
        lib.bkd_get_stat.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        lib.bkd_tree_shape.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.bkd_export_tree.argtypes = [vp, vp, vp, vp]
        lib.bkd_free.argtypes = [vp]
        lib.bkd_free.restype = None
        lib.bkd_serve_open.argtypes = [vp, i32, i64, ctypes.POINTER(vp)]
        lib.bkd_serve_submit.argtypes = [vp, vp, i64, i32, vp, vp,
                                         ctypes.POINTER(ctypes.c_int64)]
        lib.bkd_serve_step.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        lib.bkd_serve_status.argtypes = [vp, i64, ctypes.POINTER(i32)]
        lib.bkd_serve_close.argtypes = [vp]
        lib.bkd_serve_close.restype = None
        lib.bkd_outlier_scores.argtypes = [vp, i32, vp]
        lib.bkd_test_fail_alloc.argtypes = [i64]
        lib.bkd_test_host_screen.argtypes = [vp, i64, i32, i32, vp, vp, vp,
                                             vp, vp, vp, vp, vp, vp, vp]
        lib.bkd_probe_mma.argtypes = [i32, i32, vp, vp, vp, vp]
        lib.bkd_probe_umma.argtypes = [i32, i32, i32, vp, vp, vp]
        lib.bkd_last_error.restype = ctypes.c_char_p
        for f in ("bkd_build", "bkd_build_with", "bkd_query",
                  "bkd_query_static", "bkd_set_option",
                  "bkd_get_stat", "bkd_tree_shape", "bkd_export_tree",
                  "bkd_serve_open", "bkd_serve_submit", "bkd_serve_step",
                  "bkd_serve_status", "bkd_test_fail_alloc",
                  "bkd_test_host_screen",
                  "bkd_outlier_scores",
                  "bkd_probe_mma", "bkd_probe_umma"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != BKD_OK:
        raise BkdError(rc, load().bkd_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.split(".")[0] == "torch"


def _stream_for_call(stream) -> int:
    """The BKD_OPT_STREAM value that orders a call after the work queued on
    torch stream ``stream`` (which wrote its inputs).  A stream with a handle
    of its own is passed on: the call runs on it.  The legacy default stream
    has the handle 0, which the library reads as "its own stream" (not
    ordered with the default stream), so for it the host first waits for the
    stream.  Either way the call returns after its results are complete."""
    handle = int(stream.cuda_stream)
    if handle == 0:
        stream.synchronize()
    return handle


def _run_on_current_stream(tree: "Tree", device):
    import torch
    _check(load().bkd_set_option(
        tree.handle, OPTIONS["stream"],
        _stream_for_call(torch.cuda.current_stream(device))))


def _ptr(x, dtype: str, rows_cols=None):
    """(pointer, shape) of a contiguous numpy array / torch tensor."""
    if _is_torch(x):
        import torch
        want = {"f32": torch.float32, "i64": torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return x.data_ptr(), tuple(x.shape)
    want = {"f32": np.float32, "i64": np.int64}[dtype]
    if not isinstance(x, np.ndarray) or x.dtype != want \
            or not x.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous {np.dtype(want)} array")
    return x.ctypes.data, x.shape


class Tree:
    """Owning wrapper of a ``bkd_tree*`` handle."""

    def __init__(self, handle: int, keepalive=None):
        self.handle = ctypes.c_void_p(handle)
        self._keepalive = keepalive

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle and self.handle.value:
            load().bkd_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    @property
    def shape(self):
        return bkd_tree_shape(self)

    def query(self, Q, k: int, out_idx=None, out_dist=None):
        return bkd_query(self, Q, k, out_idx, out_dist)

    def stat(self, name: str) -> float:
        return bkd_get_stat(self, name)


def bkd_build(P, height: int, **options) -> Tree:
    """``bkd_build`` / ``bkd_build_with``: P is (n, d) float32."""
    lib = load()
    p, shape = _ptr(P, "f32")
    if len(shape) != 2:
        raise ValueError("P must be (n, d)")
    n, d = shape
    if _is_torch(P) and P.is_cuda:
        # the build reads P with a synchronous copy that is not ordered with
        # torch's other streams: P must be final now
        import torch
        torch.cuda.current_stream(P.device).synchronize()
    out = ctypes.c_void_p()
    if options:
        flat = []
        for key, val in options.items():
            if key not in OPTIONS:
                raise ValueError(f"unknown option {key}")
            flat += [OPTIONS[key], int(val)]
        arr = (ctypes.c_int64 * len(flat))(*flat)
        _check(lib.bkd_build_with(p, n, d, height, arr, len(options),
                                  ctypes.byref(out)))
    else:
        _check(lib.bkd_build(p, n, d, height, ctypes.byref(out)))
    return Tree(out.value)


def bkd_query(tree: Tree, Q, k: int, out_idx=None, out_dist=None):
    """``bkd_query``: returns (idx int64 (m, k), dist float32 (m, k)), on the
    same device as Q unless output buffers are given."""
    lib = load()
    q, shape = _ptr(Q, "f32")
    if len(shape) != 2:
        raise ValueError("Q must be (m, d)")
    m = shape[0]
    if out_idx is None or out_dist is None:
        if _is_torch(Q):
            import torch
            out_idx = torch.empty((m, k), dtype=torch.int64, device=Q.device)
            out_dist = torch.empty((m, k), dtype=torch.float32,
                                   device=Q.device)
        else:
            out_idx = np.empty((m, k), np.int64)
            out_dist = np.empty((m, k), np.float32)
    oi, si = _ptr(out_idx, "i64")
    od, sd = _ptr(out_dist, "f32")
    if tuple(si) != (m, k) or tuple(sd) != (m, k):
        raise ValueError("outputs must be (m, k)")
    if _is_torch(Q) and Q.is_cuda:
        _run_on_current_stream(tree, Q.device)
    _check(lib.bkd_query(tree.handle, q, m, k, oi, od))
    return out_idx, out_dist


def bkd_query_static(tree: Tree, Q, k: int, out_idx, out_dist):
    """``bkd_query_static``: the allocation-free query.  Q, out_idx and
    out_dist must be caller-allocated CUDA tensors ((m, d) float32, (m, k)
    int64, (m, k) float32); m <= BKD_STATIC_MAX_QUERIES."""
    lib = load()
    q, shape = _ptr(Q, "f32")
    oi, si = _ptr(out_idx, "i64")
    od, sd = _ptr(out_dist, "f32")
    m = shape[0]
    if tuple(si) != (m, k) or tuple(sd) != (m, k):
        raise ValueError("outputs must be (m, k)")
    if _is_torch(Q) and Q.is_cuda:
        # the call runs on the tree's stream: order it after the work that
        # wrote Q on torch's current stream
        _run_on_current_stream(tree, Q.device)
    _check(lib.bkd_query_static(tree.handle, q, m, k, oi, od))
    return out_idx, out_dist


def bkd_outlier_scores(tree: Tree, k: int, out=None, device=None):
    """``bkd_outlier_scores``: (n,) float32 mean distance of every reference
    point to its k nearest other points.  ``out`` (n,) float32 numpy array or
    torch tensor; by default a numpy array, or a CUDA tensor on ``device``."""
    lib = load()
    n = bkd_tree_shape(tree)["n"]
    if out is None:
        if device is not None:
            import torch
            out = torch.empty(n, dtype=torch.float32, device=device)
        else:
            out = np.empty(n, np.float32)
    o, shape = _ptr(out, "f32")
    if tuple(shape) != (n,):
        raise ValueError("out must be (n,)")
    if _is_torch(out) and out.is_cuda:
        _run_on_current_stream(tree, out.device)
    _check(lib.bkd_outlier_scores(tree.handle, k, o))
    return out


def bkd_set_option(tree: Tree, name: str, value: int):
    _check(load().bkd_set_option(tree.handle, OPTIONS[name], int(value)))


def bkd_get_stat(tree: Tree, name: str) -> float:
    v = ctypes.c_double()
    _check(load().bkd_get_stat(tree.handle, STATS[name], ctypes.byref(v)))
    return v.value


def bkd_tree_shape(tree: Tree) -> dict:
    n, d, h = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    ch, nc = ctypes.c_int(), ctypes.c_int()
    _check(load().bkd_tree_shape(tree.handle, ctypes.byref(n), ctypes.byref(d),
                                 ctypes.byref(h), ctypes.byref(ch),
                                 ctypes.byref(nc)))
    return {"n": n.value, "d": d.value, "height": h.value,
            "chunked": bool(ch.value), "chunks": nc.value}


def bkd_export_tree(tree: Tree):
    """(split (2^h-1,) float32, leaf_lo (2^h+1,) int64, perm (n,) int64)."""
    s = bkd_tree_shape(tree)
    L = 1 << s["height"]
    split = np.empty(max(L - 1, 1), np.float32)
    leaf_lo = np.empty(L + 1, np.int64)
    perm = np.empty(s["n"], np.int64)
    _check(load().bkd_export_tree(tree.handle, split.ctypes.data,
                                  leaf_lo.ctypes.data, perm.ctypes.data))
    return split[:L - 1], leaf_lo, perm


def bkd_free(tree: Tree):
    tree.close()


def bkd_test_fail_alloc(nth: int):
    """``bkd_test_fail_alloc``: the nth allocation from now fails (0: off)."""
    _check(load().bkd_test_fail_alloc(int(nth)))


def bkd_test_host_screen(P, height: int) -> dict:
    """``bkd_test_host_screen``: the host half of ``bkd_build`` (tree, node
    boxes, BF16 warp-screen operands and bounds) for host float32 P (n, d),
    without a GPU.  Returns numpy arrays keyed like the C arguments, plus
    ``lcap``, ``stride``, ``kh``, ``Dp``, ``tiles`` and ``tc_kh``."""
    lib = load()
    P = np.ascontiguousarray(P, np.float32)
    if P.ndim != 2:
        raise ValueError("P must be (n, d)")
    n, d = P.shape
    shape = np.zeros(8, np.int64)
    nul = ctypes.c_void_p(0)
    _check(lib.bkd_test_host_screen(P.ctypes.data, n, d, height,
                                    shape.ctypes.data, nul, nul, nul, nul,
                                    nul, nul, nul, nul, nul))
    lcap, stride, kh, nwords, Dp, tiles, tc_kh, tc_elems = (
        int(x) for x in shape)
    L = 1 << height
    out = {"split": np.empty(max(L - 1, 1), np.float32),
           "leaf_lo": np.empty(L + 1, np.int64),
           "perm": np.empty(n, np.int64),
           "box": np.empty((2 * L - 1, 2 * Dp), np.float32),
           "words": np.empty(nwords, np.uint32),
           "center": np.empty((L, d), np.float32),
           "bmax": np.empty(L, np.float32),
           "pnmax": np.empty(L, np.float32),
           "tc_words": np.empty(tc_elems, np.uint16)}
    _check(lib.bkd_test_host_screen(
        P.ctypes.data, n, d, height, shape.ctypes.data,
        *(out[key].ctypes.data for key in ("split", "leaf_lo", "perm", "box",
                                           "words", "center", "bmax",
                                           "pnmax", "tc_words"))))
    out["split"] = out["split"][:L - 1]
    out.update(lcap=lcap, stride=stride, kh=kh, Dp=Dp, tiles=tiles,
               tc_kh=tc_kh)
    return out


def bkd_probe_mma(A, Bt, C, kind: int = 0):
    """``bkd_probe_mma``: D = C + A Bt^T per instance on the warp screen
    kernel's tensor-core instruction (mma.sync m16n8k16).  A (count, 16, 16) and Bt (count, 8, 16) uint16 bf16
    bit patterns, C (count, 16, 8) float32; returns D like C."""
    A = np.ascontiguousarray(A, np.uint16)
    Bt = np.ascontiguousarray(Bt, np.uint16)
    C = np.ascontiguousarray(C, np.float32)
    count = A.shape[0]
    if A.shape != (count, 16, 16) or Bt.shape != (count, 8, 16) \
            or C.shape != (count, 16, 8):
        raise ValueError("shapes (count,16,16), (count,8,16), (count,16,8)")
    D = np.empty_like(C)
    _check(load().bkd_probe_mma(kind, count, A.ctypes.data, Bt.ctypes.data,
                                C.ctypes.data, D.ctypes.data))
    return D


def bkd_probe_umma(A, Bt):
    """``bkd_probe_umma``: D = A Bt^T per instance on the screen's
    tcgen05 path.  A (count, 128, 16 kh) and Bt (count, n, 16 kh) uint16
    bf16 bit patterns; returns D (count, 128, n) float32."""
    A = np.ascontiguousarray(A, np.uint16)
    Bt = np.ascontiguousarray(Bt, np.uint16)
    count, rows, kdim = A.shape
    n = Bt.shape[1]
    if rows != 128 or kdim % 16 or Bt.shape != (count, n, kdim):
        raise ValueError("shapes (count,128,16kh), (count,n,16kh)")
    D = np.empty((count, 128, n), np.float32)
    _check(load().bkd_probe_umma(n, kdim // 16, count, A.ctypes.data,
                                 Bt.ctypes.data, D.ctypes.data))
    return D


def bkd_last_error() -> str:
    return load().bkd_last_error().decode()


class Server:
    """``bkd_serve_*``: continuous batching over a resident tree.

        srv = Server(tree, k_max=50, max_queries=1 << 20)
        t = srv.submit(Q, k)          # queued; outputs allocated here
        while srv.step():             # one shared LazySearch round
            ...                       # submit more at any time
        idx, dist = srv.result(t)     # after status(t) == BKD_BATCH_DONE
    """

    def __init__(self, tree: Tree, k_max: int, max_queries: int):
        lib = load()
        out = ctypes.c_void_p()
        _check(lib.bkd_serve_open(tree.handle, k_max, max_queries,
                                  ctypes.byref(out)))
        self.handle = out
        self.tree = tree
        self._io = {}  # ticket -> (Q, out_idx, out_dist), kept alive

    def submit(self, Q, k: int, out_idx=None, out_dist=None) -> int:
        lib = load()
        q, shape = _ptr(Q, "f32")
        m = shape[0]
        if out_idx is None or out_dist is None:
            if _is_torch(Q):
                import torch
                out_idx = torch.empty((m, k), dtype=torch.int64,
                                      device=Q.device)
                out_dist = torch.empty((m, k), dtype=torch.float32,
                                       device=Q.device)
            else:
                out_idx = np.empty((m, k), np.int64)
                out_dist = np.empty((m, k), np.float32)
        oi, _ = _ptr(out_idx, "i64")
        od, _ = _ptr(out_dist, "f32")
        if _is_torch(Q) and Q.is_cuda:
            # the server copies Q in a later step, on the tree's stream: Q
            # must be final now (it stays unchanged until the batch is done)
            import torch
            torch.cuda.current_stream(Q.device).synchronize()
        ticket = ctypes.c_int64()
        _check(lib.bkd_serve_submit(self.handle, q, m, k, oi, od,
                                    ctypes.byref(ticket)))
        self._io[ticket.value] = (Q, out_idx, out_dist)
        return ticket.value

    def step(self) -> int:
        """One admission + round + completion pass; returns the number of
        batches not yet completed."""
        pending = ctypes.c_int64()
        _check(load().bkd_serve_step(self.handle, ctypes.byref(pending)))
        return pending.value

    def status(self, ticket: int) -> int:
        st = ctypes.c_int()
        _check(load().bkd_serve_status(self.handle, ticket, ctypes.byref(st)))
        return st.value

    def result(self, ticket: int):
        """(out_idx, out_dist) of a ticket whose status was DONE."""
        _, oi, od = self._io.pop(ticket)
        return oi, od

    def close(self):
        if self.handle and self.handle.value:
            load().bkd_serve_close(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bkd_serve_open(tree: Tree, k_max: int, max_queries: int) -> Server:
    """``bkd_serve_open``."""
    return Server(tree, k_max, max_queries)


def bkd_serve_submit(server: Server, Q, k: int, out_idx=None,
                     out_dist=None) -> int:
    """``bkd_serve_submit``: returns the ticket."""
    return server.submit(Q, k, out_idx, out_dist)


def bkd_serve_step(server: Server) -> int:
    """``bkd_serve_step``: returns the batches not yet completed."""
    return server.step()


def bkd_serve_status(server: Server, ticket: int) -> int:
    """``bkd_serve_status``."""
    return server.status(ticket)


def bkd_serve_close(server: Server):
    """``bkd_serve_close``."""
    server.close()
