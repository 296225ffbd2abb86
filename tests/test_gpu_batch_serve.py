"""Batched counting (one pass over a disjoint union of many graphs, and its
CUDA-graph plan) and the continuous-batching server, against the oracle."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1804_06926_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06926_gb300 import binding
    return binding


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_batch(b):
    Ts, ts = [], []
    for i in range(b.G):
        g = b.graph(i)
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        Ts.append(T)
        ts.append(t)
    return np.array(Ts, np.int64), np.concatenate(ts)


@pytest.mark.parametrize("cfg", [dict(), dict(small_max=-1, warp_max=8), dict(probe=2, table_cap=64)])
def test_batch_matches_oracle(B, cfg):
    ctx = B.Context(0, **cfg)
    b = gen.ba_batch(48, 100, 3000, 2, 16, seed0=17)
    T, t = oracle_batch(b)
    totals = torch.zeros(b.G, dtype=torch.int64, device="cuda")
    pv = torch.zeros(int(b.vtx_off[-1]), dtype=torch.int64, device="cuda")
    ctx.count_batch(dev(b.vtx_off), dev(b.edge_off), dev(b.row_ptr), dev(b.col), totals, pv)
    np.testing.assert_array_equal(totals.cpu().numpy(), T)
    np.testing.assert_array_equal(pv.cpu().numpy(), t)
    # host inputs and outputs
    th = np.zeros(b.G, np.int64)
    ctx.count_batch(b.vtx_off, b.edge_off, b.row_ptr, b.col, th, validate=True)
    np.testing.assert_array_equal(th, T)


def test_batch_mixed_with_empty_graphs(B):
    ctx = B.Context(0)
    graphs = [gen.from_pairs(3, [], []), gen.rmat(9, 8, seed=1), gen.from_pairs(1, [], []),
              gen.grid(10, 12, seed=0), gen.er(1024, 8192, seed=2)]
    vo = np.cumsum([0] + [g.n for g in graphs]).astype(np.int64)
    eo = np.cumsum([0] + [g.nnz for g in graphs]).astype(np.int64)
    rp = np.concatenate([g.row_ptr[:-1] + eo[i] for i, g in enumerate(graphs)] + [eo[-1:]]).astype(np.int64)
    col = np.concatenate([g.col for g in graphs]).astype(np.int32)
    totals = np.zeros(len(graphs), np.int64)
    pv = np.zeros(int(vo[-1]), np.int64)
    ctx.count_batch(vo, eo, rp, col, totals, pv, validate=True)
    for i, g in enumerate(graphs):
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        assert totals[i] == T
        np.testing.assert_array_equal(pv[vo[i]:vo[i + 1]], t)


def test_batch_plan_replays(B):
    ctx = B.Context(0)
    b = gen.ba_batch(32, 100, 2000, 2, 12, seed0=3)
    T, t = oracle_batch(b)
    vo, eo, rp, col = dev(b.vtx_off), dev(b.edge_off), dev(b.row_ptr), dev(b.col)
    totals = torch.zeros(b.G, dtype=torch.int64, device="cuda")
    pv = torch.zeros(int(b.vtx_off[-1]), dtype=torch.int64, device="cuda")
    plan = ctx.batch_plan(vo, eo, rp, col, totals, pv)
    for _ in range(3):
        totals.fill_(-1)
        pv.fill_(-1)
        plan.launch()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(totals.cpu().numpy(), T)
        np.testing.assert_array_equal(pv.cpu().numpy(), t)
    plan.close()


# ---------------------------------------------------------------- serving
def serving_mix(k, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        if rng.random() < 0.5:
            out.append(gen.rmat(int(rng.integers(8, 14)), 16, seed=int(rng.integers(0, 1 << 30))))
        else:
            out.append(gen.ba(int(rng.integers(100, 5000)), int(rng.integers(2, 17)), seed=int(rng.integers(0, 1 << 30))))
    return out


def test_server_mix_equals_alone(B):
    graphs = serving_mix(24, seed=1)
    expect = [oracle.count(g.n, g.row_ptr, g.col) for g in graphs]
    # alone: one slot, one request at a time
    srv = B.Server(slots=1, per_vertex=True)
    alone = []
    for g in graphs:
        tk = srv.submit(g.n, g.row_ptr, g.col)
        alone.append(srv.wait(tk, 60000))
    srv.close()
    # mixed: 8 slots, all submitted at once, some repeated keys; once with every
    # request on its own slot, once with small requests fused into batches
    for fuse in (1, 32):
        srv = B.Server(slots=8, per_vertex=True, batch_graphs=fuse)
        tickets = [srv.submit(g.n, g.row_ptr, g.col, key=1000 + (i % 12)) for i, g in enumerate(graphs[:12])]
        tickets += [srv.submit(g.n, g.row_ptr, g.col) for g in graphs[12:]]
        mixed = [srv.wait(tk, 60000) for tk in tickets]
        st = srv.stats()
        srv.close()
        for (T, t), a, m in zip(expect, alone, mixed):
            assert a["status"] == 0 and m["status"] == 0
            assert a["total"] == T == m["total"]
            np.testing.assert_array_equal(a["per_vertex"], t)
            np.testing.assert_array_equal(m["per_vertex"], t)
        assert st["finished"] == len(graphs)
        if fuse == 1:
            assert st["peak_inflight"] >= 2 and st["batches"] == 0


def test_server_fuses_small_requests(B):
    """Small requests queued together run as fused batches; every result stays
    exact, including graphs without edges and a repeated graph."""
    graphs = serving_mix(30, seed=4) + [gen.from_pairs(7, [], []), gen.from_pairs(1, [], [])]
    graphs.append(graphs[0])
    # a larger request first holds the only slot while the small ones queue up
    graphs.insert(0, gen.rmat(17, 16, seed=2))
    expect = [oracle.count(g.n, g.row_ptr, g.col) for g in graphs]
    srv = B.Server(slots=1, per_vertex=True, batch_graphs=8, batch_nnz=1 << 19)
    tickets = [srv.submit(g.n, g.row_ptr, g.col) for g in graphs]
    res = [srv.wait(tk, 60000) for tk in tickets]
    st = srv.stats()
    srv.close()
    for (T, t), r in zip(expect, res):
        assert r["status"] == 0 and r["total"] == T
        np.testing.assert_array_equal(r["per_vertex"], t)
    assert st["batches"] >= 2 and st["finished"] == len(graphs)


def test_server_cache_hits_and_edge_lists(B):
    srv = B.Server(slots=4)
    g = gen.rmat(12, 16, seed=3, keep_pairs=True)
    T = oracle.count(g.n, g.row_ptr, g.col)[0]
    r1 = srv.wait(srv.submit(g.n, g.row_ptr, g.col, key=42))
    r2 = srv.wait(srv.submit(g.n, g.row_ptr, g.col, key=42))
    r3 = srv.wait(srv.submit_edges(g.n, g.src, g.dst))
    assert r1["total"] == r2["total"] == r3["total"] == T
    assert not r1["cache_hit"] and r2["cache_hit"]
    srv.close()


def test_server_budget_admission(B):
    g = gen.rmat(12, 16, seed=5)
    T = oracle.count(g.n, g.row_ptr, g.col)[0]
    # a budget below one request's estimate refuses it
    srv = B.Server(slots=4, hbm_budget_bytes=1 << 20)
    r = srv.wait(srv.submit(g.n, g.row_ptr, g.col))
    assert r["status"] == B.TC_ERR_BUDGET
    srv.close()
    # a budget for about two requests admits them a few at a time, all exact
    srv = B.Server(slots=8, hbm_budget_bytes=64 << 20)
    tks = [srv.submit(g.n, g.row_ptr, g.col) for _ in range(10)]
    res = [srv.wait(t) for t in tks]
    assert all(x["status"] == 0 and x["total"] == T for x in res)
    assert srv.stats()["peak_inflight_bytes"] <= 64 << 20
    srv.close()


def test_server_poll_and_timeout(B):
    srv = B.Server(slots=2)
    g = gen.rmat(14, 16, seed=9)
    tk = srv.submit(g.n, g.row_ptr, g.col)
    t0 = time.time()
    res = None
    while res is None and time.time() - t0 < 60:
        res = srv.poll(tk)
        time.sleep(0.001)
    assert res is not None and res["total"] == oracle.count(g.n, g.row_ptr, g.col)[0]
    assert srv.release(tk) == 0
    with pytest.raises(B.TCError):
        srv.wait(tk, 10)  # released: unknown ticket
    srv.close()


def test_server_fused_totals_without_per_vertex(B):
    """Fused batches with per-vertex output off: every total exact."""
    graphs = [gen.rmat(16, 16, seed=8)] + serving_mix(20, seed=6)
    expect = [oracle.count(g.n, g.row_ptr, g.col)[0] for g in graphs]
    srv = B.Server(slots=1, per_vertex=False, batch_graphs=16)
    tickets = [srv.submit(g.n, g.row_ptr, g.col) for g in graphs]
    res = [srv.wait(tk, 60000) for tk in tickets]
    st = srv.stats()
    srv.close()
    for T, r in zip(expect, res):
        assert r["status"] == 0 and r["total"] == T and r["per_vertex"] is None
    assert st["batches"] >= 1
