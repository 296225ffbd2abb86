"""Parity at the benchmark sizes, in the launch configuration bench.py times
(default tc_config, per-vertex counts on).

* R-MAT scale 22: the oracle's total T (forward algorithm over strided row
  subsets in a spawn-started process pool) must equal the GPU total; sampled
  vertices' t(v) from the definition (adjacent pairs among N(v)) must equal
  the GPU's; sum t = 3T.
* 4096 x 4096 road-like grid: full oracle, every t(v) bit-exact.
* 4096 Barabasi-Albert graphs in one batched pass: every per-graph total
  against the oracle, per-vertex counts of sampled graphs bit-exact.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1804_06926_gb300 import gen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

# the pool is started with spawn, so no worker inherits a CUDA context
_CTX = mp.get_context("spawn")


def _rows_worker(args):
    path, n, r, stride = args
    d = np.load(path, mmap_mode="r")
    return oracle.count_rows(n, np.asarray(d["rpp"]), np.asarray(d["colp"]), r, n, stride)


def oracle_total_parallel(n, row_ptr, col, procs=None):
    """T from the oracle: orient once, then count strided row subsets in parallel."""
    rpp, colp = oracle.orient(n, row_ptr, col)
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ocsr.npz")
        np.savez(path, rpp=rpp, colp=colp)
        with _CTX.Pool(procs) as pool:
            parts = pool.map(_rows_worker, [(path, n, r, procs) for r in range(procs)])
    return int(sum(parts))


def _batch_worker(args):
    path, lo, hi = args
    d = np.load(path, mmap_mode="r")
    vo, eo, rp, col = d["vo"], d["eo"], d["rp"], d["col"]
    out = []
    for i in range(lo, hi):
        v0, v1, e0, e1 = int(vo[i]), int(vo[i + 1]), int(eo[i]), int(eo[i + 1])
        T, _ = oracle.count(v1 - v0, np.asarray(rp[v0:v1 + 1]) - e0, np.asarray(col[e0:e1]), per_vertex=False)
        out.append(T)
    return out


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06926_gb300 import binding
    return binding


def gpu_count(ctx, g):
    o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    ctx.count(o, tot, pv)
    torch.cuda.synchronize()
    o.free()
    return int(tot.item()), pv.cpu().numpy()


def test_rmat22_total_and_sampled_vertices(B):
    g = gen.rmat(22, 16, seed=0)
    ctx = B.Context(0)
    T, t = gpu_count(ctx, g)
    assert int(t.sum()) == 3 * T
    assert T == oracle_total_parallel(g.n, g.row_ptr, g.col)
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(0)
    cand = np.nonzero((deg > 0) & (deg <= 3000))[0]
    sample = list(rng.choice(cand, 300, replace=False))
    sample += list(np.argsort(deg)[-20000:][::2000])  # a few high-degree vertices as well
    for v in sample:
        assert oracle.vertex_triangles(g.n, g.row_ptr, g.col, int(v)) == t[v], v


def test_grid4096_full(B):
    g = gen.grid(4096, 4096, seed=0)
    ctx = B.Context(0)
    T, t = gpu_count(ctx, g)
    To, to = oracle.count(g.n, g.row_ptr, g.col)
    assert T == To
    np.testing.assert_array_equal(t, to)


def test_ba_batch4096(B):
    b = gen.ba_batch(4096, 100, 20000, 2, 16, seed0=0)
    ctx = B.Context(0)
    totals = torch.zeros(b.G, dtype=torch.int64, device="cuda")
    pv = torch.zeros(int(b.vtx_off[-1]), dtype=torch.int64, device="cuda")
    dev = [torch.from_numpy(x).cuda() for x in (b.vtx_off, b.edge_off, b.row_ptr, b.col)]
    ctx.count_batch(*dev, totals, pv)
    torch.cuda.synchronize()
    T_gpu = totals.cpu().numpy()
    pv_gpu = pv.cpu().numpy()
    procs = max(1, min(16, os.cpu_count() or 1))
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "batch.npz")
        np.savez(path, vo=b.vtx_off, eo=b.edge_off, rp=b.row_ptr, col=b.col)
        cuts = np.linspace(0, b.G, procs + 1).astype(int)
        with _CTX.Pool(procs) as pool:
            parts = pool.map(_batch_worker, [(path, int(cuts[i]), int(cuts[i + 1])) for i in range(procs)])
    T_ref = np.array([x for p in parts for x in p], np.int64)
    np.testing.assert_array_equal(T_gpu, T_ref)
    for i in (0, 1, 777, 2048, 4095):
        gi = b.graph(i)
        _, t = oracle.count(gi.n, gi.row_ptr, gi.col)
        np.testing.assert_array_equal(pv_gpu[b.vtx_off[i]:b.vtx_off[i + 1]], t)
