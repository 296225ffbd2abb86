"""Multi-rank logic on CPU (gloo, world size 2): partitions of a batch and of
one graph's rows, and the all-reduce that combines partial counts.  The
partial counts come from the oracle, so no GPU is needed."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1804_06926_gb300 import dist as tdist
from paper_1804_06926_gb300 import gen


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_graph_ranges_cover_and_balance():
    b = gen.ba_batch(64, 100, 3000, 2, 12, seed0=1)
    rs = tdist.graph_ranges(b.edge_off, 4)
    assert rs[0][0] == 0 and rs[-1][1] == b.G
    assert all(rs[i][1] == rs[i + 1][0] for i in range(3))
    loads = [int(b.edge_off[hi] - b.edge_off[lo]) for lo, hi in rs]
    assert max(loads) < 0.5 * sum(loads)
    assert tdist.graph_ranges(b.edge_off, 1) == [(0, b.G)]


def test_row_ranges_balance_work():
    w = np.random.default_rng(0).pareto(1.5, 10000)
    rs = tdist.row_ranges(w, 3)
    assert rs[0][0] == 0 and rs[-1][1] == 10000
    parts = [w[lo:hi].sum() for lo, hi in rs]
    assert abs(sum(parts) - w.sum()) < 1e-6 * w.sum()


def _rank(rank, world, port, ret):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a batch: each rank counts its graph range, totals combined by all-reduce
        b = gen.ba_batch(24, 100, 2000, 2, 10, seed0=5)
        lo, hi = tdist.graph_ranges(b.edge_off, world)[rank]
        totals = torch.zeros(b.G, dtype=torch.int64)
        for i in range(lo, hi):
            g = b.graph(i)
            totals[i] = oracle.count(g.n, g.row_ptr, g.col, per_vertex=False)[0]
        dist.all_reduce(totals)
        # one graph: each rank counts its source-row range, (T, t) combined
        g = gen.rmat(11, 16, seed=3)
        rpp, colp = oracle.orient(g.n, g.row_ptr, g.col)
        work = np.diff(rpp).astype(np.float64) ** 2
        rlo, rhi = tdist.row_ranges(work, world)[rank]
        t = np.zeros(g.n, np.int64)
        T = oracle._load().oracle_count_rows(g.n, rpp.ctypes.data, colp.ctypes.data, rlo, rhi, 1, t.ctypes.data)
        Tt, tt = torch.tensor([T], dtype=torch.int64), torch.from_numpy(t)
        tdist.allreduce_counts(Tt, tt)
        if rank == 0:
            ret.put((totals.numpy().copy(), int(Tt.item()), tt.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_counts_equal_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    totals, T, t = res
    b = gen.ba_batch(24, 100, 2000, 2, 10, seed0=5)
    want = [oracle.count(b.graph(i).n, b.graph(i).row_ptr, b.graph(i).col, per_vertex=False)[0] for i in range(b.G)]
    assert totals.tolist() == want
    g = gen.rmat(11, 16, seed=3)
    T1, t1 = oracle.count(g.n, g.row_ptr, g.col)
    assert T == T1 and (t == t1).all()
