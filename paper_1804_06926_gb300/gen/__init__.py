"""Seeded synthetic graph generators (input data only; no part of the method).

The C side (``tcgen.c``) draws every random number from a counter-based
SplitMix64 stream keyed by (generator, seed), so a graph is a pure function of
its parameters.  Each generator returns a simple undirected graph as a CSR with
``int64 row_ptr[n+1]`` and ``int32 col[2m]`` (neighbours ascending, no loops,
no duplicates), the input format of the paper's problem statement (Sec. 3,
undirected graphs; Table 1 caption on de-duplication and both directions).

Workload recipes (the shapes of the paper's scale-free and mesh-like inputs):
  * ``er(n, m, seed)``             G(n, m)
  * ``rmat(scale, ef, seed)``      R-MAT (a, b, c, d) = (0.57, 0.19, 0.19, 0.05)
  * ``grid(R, C, seed)``           lattice + diagonals p=0.3 + 1 % long-range
  * ``ba(n, k, seed)``             Barabasi-Albert
  * ``ba_batch(G, ...)``           G BA graphs, concatenated with int64 offsets
"""
from __future__ import annotations

import ctypes
import os
import platform
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libtcgen.so")
_lib = None

_i64, _i32, _u64, _f64, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``libtcgen.so`` in place with gcc (OpenMP, portable flags)."""
    src = os.path.join(_HERE, "tcgen.c")
    stamp = _SO + ".arch"
    try:
        arch_ok = open(stamp).read().strip() == platform.machine()
    except OSError:
        arch_ok = False
    if force or not arch_ok or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        import subprocess
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name, args in {
            "tcg_er": [_i64, _i64, _u64, _i32],
            "tcg_rmat": [_i32, _i64, _f64, _f64, _f64, _u64, _i32, _i32],
            "tcg_grid": [_i64, _i64, _f64, _f64, _u64, _i32],
            "tcg_ba": [_i64, _i64, _u64, _i32],
            "tcg_ba_batch": [_i64, _i64, _i64, _i64, _i64, _u64],
            "tcg_from_pairs": [_i64, _i64, _vp, _vp, _i32],
        }.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _vp
        for name in ("tcg_n", "tcg_nnz", "tcg_npairs", "tcg_batch_count"):
            getattr(lib, name).argtypes = [_vp]
            getattr(lib, name).restype = _i64
        lib.tcg_copy_csr.argtypes = [_vp, _vp, _vp]
        lib.tcg_copy_pairs.argtypes = [_vp, _vp, _vp]
        lib.tcg_copy_batch.argtypes = [_vp, _vp, _vp]
        lib.tcg_free.argtypes = [_vp]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Simple undirected graph: CSR (both directions) plus the raw pairs it came from."""
    n: int
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [2m], ascending within each row
    src: np.ndarray | None = None  # raw int32 pairs before canonicalisation
    dst: np.ndarray | None = None

    @property
    def m(self) -> int:
        return int(self.col.shape[0] // 2)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


@dataclass
class Batch:
    """G graphs concatenated: global row_ptr offsets into col, LOCAL neighbour ids."""
    vtx_off: np.ndarray   # int64 [G+1]
    edge_off: np.ndarray  # int64 [G+1]
    row_ptr: np.ndarray   # int64 [sum n_i + 1]
    col: np.ndarray       # int32 [sum nnz_i]

    @property
    def G(self) -> int:
        return int(self.vtx_off.shape[0] - 1)

    def graph(self, i: int) -> Graph:
        v0, v1 = int(self.vtx_off[i]), int(self.vtx_off[i + 1])
        e0, e1 = int(self.edge_off[i]), int(self.edge_off[i + 1])
        return Graph(v1 - v0, (self.row_ptr[v0:v1 + 1] - e0).astype(np.int64), self.col[e0:e1].copy())


def _take(h, keep_pairs: bool) -> Graph:
    lib = _load()
    if not h:
        raise ValueError("generator rejected its parameters")
    try:
        n, nnz = lib.tcg_n(h), lib.tcg_nnz(h)
        rp = np.empty(n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        lib.tcg_copy_csr(h, rp.ctypes.data, col.ctypes.data)
        src = dst = None
        if keep_pairs:
            np_ = lib.tcg_npairs(h)
            src = np.empty(np_, np.int32)
            dst = np.empty(np_, np.int32)
            lib.tcg_copy_pairs(h, src.ctypes.data, dst.ctypes.data)
        return Graph(int(n), rp, col, src, dst)
    finally:
        lib.tcg_free(h)


def er(n: int, m: int, seed: int = 0, keep_pairs: bool = False) -> Graph:
    return _take(_load().tcg_er(n, m, seed, int(keep_pairs)), keep_pairs)


def rmat(scale: int, edge_factor: int = 16, seed: int = 0, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, relabel: bool = True, keep_pairs: bool = False) -> Graph:
    return _take(_load().tcg_rmat(scale, edge_factor, a, b, c, seed, int(relabel), int(keep_pairs)),
                 keep_pairs)


def grid(rows: int, cols: int, seed: int = 0, p_diag: float = 0.3, frac_long: float = 0.01,
         keep_pairs: bool = False) -> Graph:
    return _take(_load().tcg_grid(rows, cols, p_diag, frac_long, seed, int(keep_pairs)), keep_pairs)


def ba(n: int, k: int, seed: int = 0, keep_pairs: bool = False) -> Graph:
    return _take(_load().tcg_ba(n, k, seed, int(keep_pairs)), keep_pairs)


def from_pairs(n: int, src, dst, keep_pairs: bool = False) -> Graph:
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    return _take(_load().tcg_from_pairs(n, s.shape[0], s.ctypes.data, d.ctypes.data,
                                        int(keep_pairs)), keep_pairs)


def ba_batch(G: int, n_lo: int = 100, n_hi: int = 20000, k_lo: int = 2, k_hi: int = 16,
             seed0: int = 0) -> Batch:
    lib = _load()
    h = lib.tcg_ba_batch(G, n_lo, n_hi, k_lo, k_hi, seed0)
    if not h:
        raise ValueError("batch generator rejected its parameters")
    try:
        n, nnz, g = lib.tcg_n(h), lib.tcg_nnz(h), lib.tcg_batch_count(h)
        rp = np.empty(n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        vo = np.empty(g + 1, np.int64)
        eo = np.empty(g + 1, np.int64)
        lib.tcg_copy_csr(h, rp.ctypes.data, col.ctypes.data)
        lib.tcg_copy_batch(h, vo.ctypes.data, eo.ctypes.data)
        return Batch(vo, eo, rp, col)
    finally:
        lib.tcg_free(h)


# Named workloads (sizes of the benchmark configurations).
def workload(name: str, seed: int = 0):
    if name == "er_1024_8192":
        return er(1024, 8192, seed)
    if name == "rmat22":
        return rmat(22, 16, seed)
    if name == "grid4096":
        return grid(4096, 4096, seed)
    if name == "ba_batch4096":
        return ba_batch(4096, 100, 20000, 2, 16, seed)
    raise KeyError(name)
