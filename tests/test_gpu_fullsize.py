"""Parity at the benchmark sizes, in the launch configuration bench.py times
(default tc_config, per-vertex counts on).

* R-MAT scale 22: the oracle's T and every one of the 4,194,304 t(v)
  (forward algorithm over strided row subsets in a spawn-started process
  pool, each worker with a private per-vertex array, summed) must equal the
  GPU's bit for bit (the hubs, whose lists fill the CTA tables, included).
* 4096 x 4096 road-like grid: full oracle, every t(v) bit-exact.
* 4096 Barabasi-Albert graphs in one batched pass: every per-graph total and
  every per-vertex count of every graph against the oracle.
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
    return oracle.count_rows_pv(n, np.asarray(d["rpp"]), np.asarray(d["colp"]), r, n, stride)


def oracle_counts_parallel(n, row_ptr, col, procs=None):
    """(T, t) from the oracle: orient once, then count strided row subsets in
    parallel, each with its own per-vertex array; the parts add up exactly."""
    rpp, colp = oracle.orient(n, row_ptr, col)
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ocsr.npz")
        np.savez(path, rpp=rpp, colp=colp)
        with _CTX.Pool(procs) as pool:
            parts = pool.map(_rows_worker, [(path, n, r, procs) for r in range(procs)])
    T = int(sum(p[0] for p in parts))
    t = np.zeros(n, np.int64)
    for p in parts:
        t += p[1]
    return T, t


def _batch_worker(args):
    path, lo, hi = args
    d = np.load(path, mmap_mode="r")
    vo, eo, rp, col = d["vo"], d["eo"], d["rp"], d["col"]
    Ts, ts = [], []
    for i in range(lo, hi):
        v0, v1, e0, e1 = int(vo[i]), int(vo[i + 1]), int(eo[i]), int(eo[i + 1])
        T, t = oracle.count(v1 - v0, np.asarray(rp[v0:v1 + 1]) - e0, np.asarray(col[e0:e1]))
        Ts.append(T)
        ts.append(t)
    return Ts, (np.concatenate(ts) if ts else np.zeros(0, np.int64))


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


def test_rmat22_every_vertex(B):
    g = gen.rmat(22, 16, seed=0)
    ctx = B.Context(0)
    T, t = gpu_count(ctx, g)
    To, to = oracle_counts_parallel(g.n, g.row_ptr, g.col)
    assert T == To
    np.testing.assert_array_equal(t, to)
    assert int(t.sum()) == 3 * T


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
    T_ref = np.array([x for p in parts for x in p[0]], np.int64)
    t_ref = np.concatenate([p[1] for p in parts])
    np.testing.assert_array_equal(T_gpu, T_ref)
    assert t_ref.shape == pv_gpu.shape
    np.testing.assert_array_equal(pv_gpu, t_ref)


def test_serving_mix_rmat10_to_20(B):
    """The serving workload's request mix at its full size range: one R-MAT
    graph of every scale 10..20 (edge factor 16) and BA graphs as in the batch
    workload, submitted together to an 8-slot server (40 GB budget, small
    requests fused into batches, some keys cached and repeated) and one at a
    time to a 1-slot server; every total and every t(v) equals the oracle's
    both ways."""
    rng = np.random.default_rng(5)
    graphs = [gen.rmat(s, 16, seed=100 + s) for s in range(10, 21)]
    graphs += [gen.ba(int(rng.integers(100, 20001)), int(rng.integers(2, 17)), seed=int(rng.integers(1 << 30)))
               for _ in range(8)]
    expect = [oracle_counts_parallel(g.n, g.row_ptr, g.col) if g.m > 1_000_000 else oracle.count(g.n, g.row_ptr, g.col)
              for g in graphs]
    srv = B.Server(slots=1, per_vertex=True, batch_graphs=1)
    alone = [srv.wait(srv.submit(g.n, g.row_ptr, g.col), 600000) for g in graphs]
    srv.close()
    order = list(rng.permutation(len(graphs))) * 2
    srv = B.Server(slots=8, per_vertex=True, hbm_budget_bytes=40 << 30)
    tickets = [srv.submit(graphs[i].n, graphs[i].row_ptr, graphs[i].col, key=(1 + int(i)) if k % 3 == 0 else 0)
               for k, i in enumerate(order)]
    mixed = [srv.wait(tk, 600000) for tk in tickets]
    st = srv.stats()
    srv.close()
    for (T, t), a in zip(expect, alone):
        assert a["status"] == 0 and a["total"] == T
        np.testing.assert_array_equal(a["per_vertex"], t)
    for i, m in zip(order, mixed):
        T, t = expect[i]
        assert m["status"] == 0 and m["total"] == T
        np.testing.assert_array_equal(m["per_vertex"], t)
    assert st["finished"] == len(order) and st["peak_inflight"] >= 2
