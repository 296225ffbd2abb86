"""TEST INFRASTRUCTURE ONLY: the CPU oracle for exact triangle counting.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1804_06926_gb300`` never imports it and shares no code with it.

``tc_oracle.c`` holds the plain forward algorithm (see its header for the
paper passages it follows); ``dense.py`` holds the dense matrix formulation
(Alg. 3) for tiny graphs.  Every function here is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``: the Fig. 1/Fig. 3
worked example, brute force over triples, trace(A^3)/6, scipy's sparse A^2 o A,
closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
_vp, _i64 = ctypes.c_void_p, ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, single thread, portable flags)."""
    src = os.path.join(_HERE, "tc_oracle.c")
    stamp = _SO + ".arch"
    try:
        arch_ok = open(stamp).read().strip() == platform.machine()
    except OSError:
        arch_ok = False
    if force or not arch_ok or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, src])
        os.replace(tmp, _SO)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_canonicalize.argtypes = [_i64, _i64, _vp, _vp, _vp, _vp, _i64]
        lib.oracle_canonicalize.restype = _i64
        lib.oracle_orient.argtypes = [_i64, _vp, _vp, _vp, _vp, _i64]
        lib.oracle_orient.restype = _i64
        lib.oracle_count_rows.argtypes = [_i64, _vp, _vp, _i64, _i64, _i64, _vp]
        lib.oracle_count_rows.restype = _i64
        lib.oracle_count.argtypes = [_i64, _vp, _vp, _vp]
        lib.oracle_count.restype = _i64
        lib.oracle_vertex_triangles.argtypes = [_i64, _vp, _vp, _i64]
        lib.oracle_vertex_triangles.restype = _i64
        lib.oracle_edge_support.argtypes = [_i64, _vp, _vp, _vp]
        lib.oracle_edge_support.restype = None
        lib.oracle_list_triangles.argtypes = [_i64, _vp, _vp, _vp, _i64]
        lib.oracle_list_triangles.restype = _i64
        _lib = lib
    return _lib


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def canonicalize(n: int, src, dst):
    """Raw pairs -> (row_ptr int64[n+1], col int32[nnz]) simple undirected CSR."""
    s, d = _c32(src), _c32(dst)
    rp = np.zeros(n + 1, np.int64)
    col = np.empty(max(2 * s.shape[0], 1), np.int32)
    nnz = _load().oracle_canonicalize(n, s.shape[0], s.ctypes.data, d.ctypes.data,
                                      rp.ctypes.data, col.ctypes.data, col.shape[0])
    if nnz < 0:
        raise ValueError("vertex id out of range")
    return rp, col[:nnz].copy()


def orient(n: int, row_ptr, col):
    """Undirected CSR -> oriented CSR (rpp int64[n+1], colp int32[m])."""
    rp, c = _c64(row_ptr), _c32(col)
    rpp = np.zeros(n + 1, np.int64)
    colp = np.empty(max(c.shape[0] // 2, 1), np.int32)
    m = _load().oracle_orient(n, rp.ctypes.data, c.ctypes.data, rpp.ctypes.data,
                              colp.ctypes.data, colp.shape[0])
    if m < 0:
        raise ValueError("input is not a symmetric simple CSR")
    return rpp, colp[:m].copy()


def count_oriented(n: int, rpp, colp, per_vertex: bool = True):
    rp, c = _c64(rpp), _c32(colp)
    t = np.zeros(n, np.int64) if per_vertex else None
    T = _load().oracle_count(n, rp.ctypes.data, c.ctypes.data, t.ctypes.data if t is not None else None)
    return int(T), t


def count_rows(n: int, rpp, colp, u_begin: int, u_end: int, stride: int = 1) -> int:
    rp, c = _c64(rpp), _c32(colp)
    return int(_load().oracle_count_rows(n, rp.ctypes.data, c.ctypes.data, u_begin, u_end, stride, None))


def count_rows_pv(n: int, rpp, colp, u_begin: int, u_end: int, stride: int = 1):
    """(T_rows, t_rows): the triangles whose lowest-ranked vertex is one of the
    rows u_begin, u_begin+stride, ... < u_end, and their per-vertex counts (a
    private int64[n] array).  Summed over a partition of the rows they give the
    whole graph's (T, t), so disjoint row subsets can run in separate processes."""
    rp, c = _c64(rpp), _c32(colp)
    t = np.zeros(n, np.int64)
    T = _load().oracle_count_rows(n, rp.ctypes.data, c.ctypes.data, u_begin, u_end, stride,
                                  t.ctypes.data if n > 0 else None)
    return int(T), t


def count(n: int, row_ptr, col, per_vertex: bool = True):
    """(T, t) for a simple undirected CSR: orient, then forward-count."""
    rpp, colp = orient(n, row_ptr, col)
    return count_oriented(n, rpp, colp, per_vertex)


def count_pairs(n: int, src, dst, per_vertex: bool = True):
    """(T, t) for a raw pair list (loops/duplicates/both directions allowed)."""
    rp, col = canonicalize(n, src, dst)
    return count(n, rp, col, per_vertex)


def vertex_triangles(n: int, row_ptr, col, v: int) -> int:
    rp, c = _c64(row_ptr), _c32(col)
    return int(_load().oracle_vertex_triangles(n, rp.ctypes.data, c.ctypes.data, int(v)))


def edge_support(n: int, row_ptr, col) -> np.ndarray:
    """Triangles containing each edge, per entry of the undirected CSR."""
    rp, c = _c64(row_ptr), _c32(col)
    sup = np.zeros(max(c.shape[0], 1), np.int64)
    _load().oracle_edge_support(n, rp.ctypes.data, c.ctypes.data, sup.ctypes.data)
    return sup[:c.shape[0]]


def list_triangles(n: int, row_ptr, col) -> np.ndarray:
    """All triangles as rows (u, v, w) in rank order (forward algorithm)."""
    rpp, colp = orient(n, row_ptr, col)
    T, _ = count_oriented(n, rpp, colp, per_vertex=False)
    tri = np.zeros((max(T, 1), 3), np.int32)
    got = _load().oracle_list_triangles(n, _c64(rpp).ctypes.data, _c32(colp).ctypes.data, tri.ctypes.data, T)
    assert got == T
    return tri[:T]


def count_labelled(n: int, row_ptr, col, labels, query) -> int:
    """Triangles whose label multiset is `query`: list every triangle, check its labels."""
    tri = list_triangles(n, row_ptr, col)
    if tri.shape[0] == 0:
        return 0
    lab = np.asarray(labels)[tri]
    lab.sort(axis=1)
    return int((lab == np.sort(np.asarray(query))).all(axis=1).sum())
