"""Thin ctypes binding of ``libtc.so`` (the C ABI of ``include/tc.h``).

Functions keep the C names and only marshal arguments; every step of the
method runs in the CUDA library.  There is no CPU fallback: importing this
module on a machine without the built library raises.

The helpers at the bottom (``Context``, ``Server``) accept torch tensors
(device memory, torch streams) or numpy arrays (host memory) and pass their
raw pointers through.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

_lib = None

TC_OK, TC_PENDING = 0, 1
TC_ERR_INVALID_ARG, TC_ERR_INVALID_GRAPH, TC_ERR_OOM = -1, -2, -3
TC_ERR_BUDGET, TC_ERR_TIMEOUT, TC_ERR_CUDA, TC_ERR_NOT_FOUND = -4, -5, -6, -7
TC_ERR_DEVICE = -8
TC_DEVERR_PROBE, TC_DEVERR_BOUNDS, TC_DEVERR_DIRTY, TC_DEVERR_WAIT = 0x1, 0x2, 0x4, 0x8
TC_IN_DEVICE, TC_IN_HOST, TC_VALIDATE = 0x0, 0x1, 0x2

STATUS_NAMES = {0: "TC_OK", 1: "TC_PENDING", -1: "TC_ERR_INVALID_ARG", -2: "TC_ERR_INVALID_GRAPH",
                -3: "TC_ERR_OOM", -4: "TC_ERR_BUDGET", -5: "TC_ERR_TIMEOUT", -6: "TC_ERR_CUDA",
                -7: "TC_ERR_NOT_FOUND", -8: "TC_ERR_DEVICE"}


class tc_graph(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("src", C.c_void_p), ("dst", C.c_void_p), ("flags", C.c_uint32)]


class tc_config(C.Structure):
    _fields_ = [("small_max", C.c_int32), ("warp_max", C.c_int32), ("table_cap", C.c_int32),
                ("probe", C.c_int32), ("cta_threads", C.c_int32), ("chunk", C.c_int32),
                ("bitmap_bits", C.c_int32), ("direct_span", C.c_int32), ("merge_ratio", C.c_int32),
                ("merge_max", C.c_int32), ("stage", C.c_int32), ("small_lanes", C.c_int32),
                ("reserved", C.c_int32 * 4)]


class tc_ocsr_view(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("bytes", C.c_int64)]


class tc_batch(C.Structure):
    _fields_ = [("G", C.c_int64), ("vtx_off", C.c_void_p), ("edge_off", C.c_void_p),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("flags", C.c_uint32)]


class tc_server_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("slots", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("per_vertex", C.c_int32), ("batch_graphs", C.c_int32), ("batch_nnz", C.c_int64),
                ("reserved", C.c_int32 * 4)]


class tc_result(C.Structure):
    _fields_ = [("status", C.c_int), ("total", C.c_int64), ("n", C.c_int64),
                ("per_vertex", C.POINTER(C.c_int64)), ("submit_to_done_ms", C.c_double),
                ("queue_ms", C.c_double), ("cache_hit", C.c_int32)]


TRACE_PHASES = ("degree", "validate", "orient_count", "orient_scan", "orient_scatter", "pivot_count",
                "pivot_scan", "pivot_scatter", "items", "count_small", "count_warp", "count_cta", "edge_sort",
                "count_init", "rank", "row_sort", "count_merge", "fused")


class tc_trace(C.Structure):
    _fields_ = [("launches", C.c_int64), ("phase_ms", C.c_double * 20), ("phase_calls", C.c_int32 * 20)]


class tc_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("finished", C.c_int64),
                ("cache_hits", C.c_int64), ("evictions", C.c_int64), ("resident_bytes", C.c_int64),
                ("peak_inflight_bytes", C.c_int64), ("peak_inflight", C.c_int32),
                ("batches", C.c_int64), ("batched_requests", C.c_int64)]


_vp, _P = C.c_void_p, C.POINTER
_SIGS = {
    "tc_ctx_create": (C.c_int, [C.c_int, _P(tc_config), _P(_vp)]),
    "tc_ctx_destroy": (None, [_vp]),
    "tc_last_error": (C.c_char_p, [_vp]),
    "tc_ctx_set_config": (C.c_int, [_vp, _P(tc_config)]),
    "tc_ctx_get_config": (C.c_int, [_vp, _P(tc_config)]),
    "tc_ctx_set_trace": (C.c_int, [_vp, C.c_int]),
    "tc_ctx_read_trace": (C.c_int, [_vp, _P(tc_trace)]),
    "tc_check": (C.c_int, [_vp, _P(C.c_uint32), _vp]),
    "tc_build_oriented_csr": (C.c_int, [_vp, _P(tc_graph), _P(_vp), _vp]),
    "tc_count": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "tc_count_graph": (C.c_int, [_vp, _P(tc_graph), _vp, _vp, _vp]),
    "tc_count_shard": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    "tc_clustering": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tc_edge_support": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, _vp, _vp]),
    "tc_masked_product": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "tc_count_labelled": (C.c_int, [_vp, _P(tc_graph), _vp, _vp, _vp, _vp]),
    "tc_ocsr_get_view": (C.c_int, [_vp, _P(tc_ocsr_view)]),
    "tc_ocsr_copy": (C.c_int, [_vp, _vp, _vp, _vp]),
    "tc_ocsr_free": (None, [_vp]),
    "tc_ocsr_release": (None, [_vp, _vp]),
    "tc_count_batch": (C.c_int, [_vp, _P(tc_batch), _vp, _vp, _vp]),
    "tc_batch_plan_create": (C.c_int, [_vp, _P(tc_batch), _vp, _vp, _vp, _P(_vp)]),
    "tc_batch_plan_launch": (C.c_int, [_vp, _vp]),
    "tc_batch_plan_destroy": (None, [_vp]),
    "tc_server_create": (C.c_int, [_P(tc_server_config), _P(tc_config), _P(_vp)]),
    "tc_server_destroy": (None, [_vp]),
    "tc_submit": (C.c_int, [_vp, _P(tc_graph), C.c_uint64, _P(C.c_uint64)]),
    "tc_poll": (C.c_int, [_vp, C.c_uint64, _P(tc_result)]),
    "tc_wait": (C.c_int, [_vp, C.c_uint64, C.c_int64, _P(tc_result)]),
    "tc_release": (C.c_int, [_vp, C.c_uint64]),
    "tc_server_get_stats": (C.c_int, [_vp, _P(tc_server_stats)]),
    "tc_orient_noalloc": (C.c_int, [C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp]),
}

TC_NOALLOC_MAX_VERTICES = 1 << 24

# names the header declares (checked against the exports by the CPU tests)
EXPORTS = tuple(_SIGS)


def debug_requested() -> bool:
    """TC_LIBRARY=debug selects the TC_DEBUG build (bounds-checked kernels)."""
    return os.environ.get("TC_LIBRARY", "") == "debug"


def library_path() -> str:
    return _build.DEBUG_LIB if debug_requested() else _build.LIB


def load(build_if_missing: bool = True):
    """Load libtc.so, or libtc_debug.so when TC_LIBRARY=debug (building it with
    nvcc if it is missing or stale)."""
    global _lib
    if _lib is None:
        dbg = debug_requested()
        path = _build.DEBUG_LIB if dbg else _build.LIB
        if build_if_missing:
            path = _build.build(debug=dbg)
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _fn(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    return call


for _name in _SIGS:
    globals()[_name] = _fn(_name)


class TCError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


# --------------------------------------------------------------------------- helpers
def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _is_host(x):
    if isinstance(x, np.ndarray):
        return True
    return not x.is_cuda


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_config(**kw) -> tc_config:
    c = tc_config()
    for k, v in kw.items():
        if v is not None:
            setattr(c, k, int(v))
    return c


class OCSR:
    """Library-owned oriented CSR (tc_ocsr handle)."""

    def __init__(self, ctx: "Context", handle):
        self.ctx = ctx
        self.handle = handle

    def view(self) -> tc_ocsr_view:
        v = tc_ocsr_view()
        _check(self.ctx, tc_ocsr_get_view(self.handle, C.byref(v)))
        return v

    def copy_to_host(self):
        v = self.view()
        rp = np.empty(v.n + 1, np.int64)
        col = np.empty(max(v.m, 1), np.int32)
        _check(self.ctx, tc_ocsr_copy(self.handle, rp.ctypes.data, col.ctypes.data, _stream_ptr(None)))
        return rp, col[:v.m]

    def free(self):
        if self.handle:
            tc_ocsr_free(self.handle)
            self.handle = None

    def release(self, stream=None):
        if self.handle:
            tc_ocsr_release(self.handle, _stream_ptr(stream))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _check(ctx, st):
    if st != TC_OK:
        msg = tc_last_error(ctx.handle).decode() if ctx is not None and ctx.handle else ""
        raise TCError(st, msg)
    return st


class Context:
    """tc_ctx with torch/numpy-facing wrappers of the ABI calls."""

    def __init__(self, device: int = 0, **cfg):
        self.handle = _vp()
        self.device = device
        st = tc_ctx_create(device, C.byref(make_config(**cfg)), C.byref(self.handle))
        if st != TC_OK:
            raise TCError(st, "tc_ctx_create")

    def set_config(self, **cfg):
        _check(self, tc_ctx_set_config(self.handle, C.byref(make_config(**cfg))))

    def get_config(self) -> dict:
        c = tc_config()
        _check(self, tc_ctx_get_config(self.handle, C.byref(c)))
        return {k: getattr(c, k) for k, _ in tc_config._fields_ if k != "reserved"}

    def set_trace(self, on: bool = True):
        _check(self, tc_ctx_set_trace(self.handle, int(on)))

    def read_trace(self) -> dict:
        """Summed device ms per phase and the number of kernel launches since the last read."""
        t = tc_trace()
        _check(self, tc_ctx_read_trace(self.handle, C.byref(t)))
        return {"launches": t.launches,
                "phase_ms": {n: t.phase_ms[i] for i, n in enumerate(TRACE_PHASES)},
                "phase_calls": {n: t.phase_calls[i] for i, n in enumerate(TRACE_PHASES)}}

    def close(self):
        if self.handle:
            tc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- build ------------------------------------------------------------
    def build(self, n, row_ptr, col, stream=None, validate=False) -> OCSR:
        """CSR input: torch device tensors, or numpy arrays (host, copied in)."""
        g = tc_graph()
        g.n, g.nnz = int(n), int(col.shape[0])
        g.row_ptr, g.col = _ptr(row_ptr), _ptr(col)
        g.flags = (TC_IN_HOST if _is_host(row_ptr) else 0) | (TC_VALIDATE if validate else 0)
        h = _vp()
        _check(self, tc_build_oriented_csr(self.handle, C.byref(g), C.byref(h), _stream_ptr(stream)))
        return OCSR(self, h)

    def build_edges(self, n, src, dst, stream=None) -> OCSR:
        g = tc_graph()
        g.n, g.nnz = int(n), int(src.shape[0])
        g.src, g.dst = _ptr(src), _ptr(dst)
        g.flags = TC_IN_HOST if _is_host(src) else 0
        h = _vp()
        _check(self, tc_build_oriented_csr(self.handle, C.byref(g), C.byref(h), _stream_ptr(stream)))
        return OCSR(self, h)

    def check(self, stream=None) -> int:
        """Synchronise, read and clear the device check word; raises TCError
        (TC_ERR_DEVICE) if a device-side check failed since the last call."""
        bits = C.c_uint32(0)
        st = tc_check(self.handle, C.byref(bits), _stream_ptr(stream))
        if st != TC_OK:
            msg = tc_last_error(self.handle).decode()
            raise TCError(st, msg)
        return bits.value

    # -- count ------------------------------------------------------------
    def count(self, o: OCSR, total=None, per_vertex=None, stream=None):
        """total / per_vertex: int64 torch tensors (device) or numpy arrays (host)."""
        _check(self, tc_count(self.handle, o.handle, _ptr(total), _ptr(per_vertex), _stream_ptr(stream)))
        return total, per_vertex

    def count_graph(self, n, row_ptr, col, total, per_vertex=None, stream=None, validate=False):
        """Build and count in one call (tc_count_graph): a graph small enough
        for one CTA's shared memory takes one fused kernel launch, any other the
        build + count path.  Inputs as in build(), outputs as in count()."""
        g = tc_graph()
        g.n, g.nnz = int(n), int(col.shape[0])
        g.row_ptr, g.col = _ptr(row_ptr), _ptr(col)
        g.flags = (TC_IN_HOST if _is_host(row_ptr) else 0) | (TC_VALIDATE if validate else 0)
        _check(self, tc_count_graph(self.handle, C.byref(g), _ptr(total), _ptr(per_vertex), _stream_ptr(stream)))
        return total, per_vertex

    def count_shard(self, o: OCSR, shard, nshards, total=None, per_vertex=None, stream=None):
        """Partial counts of one shard; summed over all shards they equal count()."""
        _check(self, tc_count_shard(self.handle, o.handle, int(shard), int(nshards), _ptr(total), _ptr(per_vertex),
                                    _stream_ptr(stream)))
        return total, per_vertex

    def clustering(self, o: OCSR, total, per_vertex, local=None, stream=None):
        """(transitivity, wedges); fills `local` (n doubles) when given."""
        tr = C.c_double(0.0)
        w = C.c_int64(0)
        _check(self, tc_clustering(self.handle, o.handle, _ptr(total), _ptr(per_vertex), _ptr(local),
                                   C.addressof(tr), C.addressof(w), _stream_ptr(stream)))
        return tr.value, w.value

    def edge_support(self, o: OCSR, support=None, triangles=None, stream=None) -> int:
        """Number of triangles; fills support (m int64) and up to len(triangles) // 3 triples."""
        cnt = C.c_int64(0)
        cap = 0 if triangles is None else int(triangles.shape[0]) // 3
        _check(self, tc_edge_support(self.handle, o.handle, _ptr(support), _ptr(triangles), cap, C.addressof(cnt),
                                     _stream_ptr(stream)))
        return cnt.value

    def masked_product(self, o: OCSR, c, stream=None) -> int:
        """Per-edge entries of the masked product C = A o (LU) (Alg. 3); returns their sum T."""
        tot = C.c_int64(0)
        _check(self, tc_masked_product(self.handle, o.handle, _ptr(c), C.addressof(tot), _stream_ptr(stream)))
        return tot.value

    def count_labelled(self, n, row_ptr, col, labels, query, stream=None) -> int:
        """Triangles whose vertex labels are the multiset `query` (device CSR and labels)."""
        g = tc_graph()
        g.n, g.nnz = int(n), int(col.shape[0])
        g.row_ptr, g.col = _ptr(row_ptr), _ptr(col)
        q = (C.c_int32 * 3)(*[int(x) for x in query])
        tot = C.c_int64(0)
        _check(self, tc_count_labelled(self.handle, C.byref(g), _ptr(labels), q, C.addressof(tot),
                                       _stream_ptr(stream)))
        return tot.value

    def count_batch(self, vtx_off, edge_off, row_ptr, col, totals, per_vertex=None, stream=None, validate=False):
        b = tc_batch()
        b.G = int(vtx_off.shape[0] - 1)
        b.vtx_off, b.edge_off, b.row_ptr, b.col = _ptr(vtx_off), _ptr(edge_off), _ptr(row_ptr), _ptr(col)
        b.flags = (TC_IN_HOST if _is_host(row_ptr) else 0) | (TC_VALIDATE if validate else 0)
        _check(self, tc_count_batch(self.handle, C.byref(b), _ptr(totals), _ptr(per_vertex), _stream_ptr(stream)))
        return totals, per_vertex

    def batch_plan(self, vtx_off, edge_off, row_ptr, col, totals, per_vertex=None, stream=None):
        b = tc_batch()
        b.G = int(vtx_off.shape[0] - 1)
        b.vtx_off, b.edge_off, b.row_ptr, b.col = _ptr(vtx_off), _ptr(edge_off), _ptr(row_ptr), _ptr(col)
        b.flags = 0
        h = _vp()
        _check(self, tc_batch_plan_create(self.handle, C.byref(b), _ptr(totals), _ptr(per_vertex),
                                          _stream_ptr(stream), C.byref(h)))
        return BatchPlan(h, keep=(vtx_off, edge_off, row_ptr, col, totals, per_vertex))


class BatchPlan:
    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep  # the captured graph reads these buffers

    def launch(self, stream=None):
        st = tc_batch_plan_launch(self.handle, _stream_ptr(stream))
        if st != TC_OK:
            raise TCError(st, "tc_batch_plan_launch")

    def close(self):
        if self.handle:
            tc_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """tc_server: continuous batching of count requests (host CSR inputs)."""

    def __init__(self, device=0, slots=8, hbm_budget_bytes=40 << 30, per_vertex=False, batch_graphs=0,
                 batch_nnz=0, **cfg):
        sc = tc_server_config()
        sc.device, sc.slots, sc.hbm_budget_bytes, sc.per_vertex = device, slots, hbm_budget_bytes, int(per_vertex)
        sc.batch_graphs, sc.batch_nnz = int(batch_graphs), int(batch_nnz)
        self.handle = _vp()
        st = tc_server_create(C.byref(sc), C.byref(make_config(**cfg)), C.byref(self.handle))
        if st != TC_OK:
            raise TCError(st, "tc_server_create")
        self.per_vertex = per_vertex

    def submit(self, n, row_ptr, col, key=0, validate=False) -> int:
        g = tc_graph()
        g.n, g.nnz = int(n), int(col.shape[0])
        g.row_ptr, g.col = _ptr(row_ptr), _ptr(col)
        g.flags = TC_IN_HOST | (TC_VALIDATE if validate else 0)
        t = C.c_uint64()
        st = tc_submit(self.handle, C.byref(g), int(key), C.byref(t))
        if st != TC_OK:
            raise TCError(st, "tc_submit")
        return t.value

    def submit_edges(self, n, src, dst, key=0) -> int:
        g = tc_graph()
        g.n, g.nnz = int(n), int(src.shape[0])
        g.src, g.dst = _ptr(src), _ptr(dst)
        g.flags = TC_IN_HOST
        t = C.c_uint64()
        st = tc_submit(self.handle, C.byref(g), int(key), C.byref(t))
        if st != TC_OK:
            raise TCError(st, "tc_submit")
        return t.value

    @staticmethod
    def _result(r: tc_result):
        pv = None
        if r.per_vertex:
            pv = np.ctypeslib.as_array(r.per_vertex, shape=(r.n,)).copy()
        return {"status": r.status, "total": r.total, "per_vertex": pv, "latency_ms": r.submit_to_done_ms,
                "queue_ms": r.queue_ms, "cache_hit": bool(r.cache_hit)}

    def poll(self, ticket):
        r = tc_result()
        st = tc_poll(self.handle, ticket, C.byref(r))
        if st == TC_PENDING:
            return None
        if st not in (TC_OK,) and r.status == TC_PENDING:
            raise TCError(st, "tc_poll")
        return self._result(r)

    def wait(self, ticket, timeout_ms=60000):
        r = tc_result()
        st = tc_wait(self.handle, ticket, int(timeout_ms), C.byref(r))
        if st == TC_ERR_TIMEOUT:
            raise TCError(st, "tc_wait")
        if st == TC_ERR_NOT_FOUND:
            raise TCError(st, "tc_wait")
        return self._result(r)

    def release(self, ticket):
        return tc_release(self.handle, ticket)

    def stats(self) -> dict:
        s = tc_server_stats()
        tc_server_get_stats(self.handle, C.byref(s))
        return {k: getattr(s, k) for k, _ in tc_server_stats._fields_}

    def close(self):
        if self.handle:
            tc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
