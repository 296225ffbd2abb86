"""Multi-rank logic on CPU (gloo, world size 2): the split of a batch by
graph ranges, the split of one graph's work lists that tc_count_shard applies
(shard k of K takes the k-th contiguous 1/K of each list), and the all-reduce
that combines partial counts.  The partial counts come from the oracle's
oriented lists, so no GPU is needed."""
import os
import socket

import numpy as np
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


def test_shard_bounds_cover_every_unit_once():
    for n_all in (0, 1, 2, 7, 1000, 2 ** 31 + 5):
        for K in (1, 2, 3, 7, 8):
            b = [tdist.shard_bounds(n_all, k, K) for k in range(K)]
            assert b[0][0] == 0 and b[-1][1] == n_all
            assert all(b[k][1] == b[k + 1][0] for k in range(K - 1))
            assert all(lo <= hi for lo, hi in b)
            assert max(hi - lo for lo, hi in b) - min(hi - lo for lo, hi in b) <= 1


def host_work_lists(n, rpp, colp, small_max=8, warp_max=128, chunk=512, table_cap=1024):
    """The partition of tc_build_oriented_csr, restated on the host: every
    oriented edge (u, v) is skipped (d+(u) <= 1 or d+(v) = 0), merged by the
    thread of its source row (max(d+) <= small_max), or given to the endpoint
    with the longer list as pivot (u on ties); pivots with d+ <= warp_max get
    items of `chunk` partners, longer ones items of (table segment, 2*chunk
    partners).  Returns (small rows, warp items, CTA items); an item is
    (p, segment, [partners])."""
    dp = np.diff(rpp)
    partners = {}
    small_rows = []
    for u in range(n):
        if 2 <= dp[u] <= small_max:
            small_rows.append(u)
        for v in colp[rpp[u]:rpp[u + 1]]:
            a, b = dp[u], dp[v]
            if a <= 1 or b == 0 or max(a, b) <= small_max:
                continue
            p, q = (u, int(v)) if a >= b else (int(v), u)
            partners.setdefault(p, []).append(q)
    warp, cta = [], []
    for p in sorted(partners):
        qs = partners[p]
        if dp[p] <= warp_max:
            warp += [(p, 0, qs[i:i + chunk]) for i in range(0, len(qs), chunk)]
        else:
            for sg in range((dp[p] + table_cap - 1) // table_cap):
                cta += [(p, sg, qs[i:i + 2 * chunk]) for i in range(0, len(qs), 2 * chunk)]
    return small_rows, warp, cta


def count_share(n, rpp, colp, shard, nshards, small_max=8, table_cap=1024):
    """(T, t) of one shard: its slice of each work list, counted edge by edge."""
    small_rows, warp, cta = host_work_lists(n, rpp, colp, small_max=small_max, table_cap=table_cap)
    dp = np.diff(rpp)
    T, t = 0, np.zeros(n, np.int64)

    def edge(p, q, keys):
        nonlocal T
        common = np.intersect1d(keys, colp[rpp[q]:rpp[q + 1]], assume_unique=True)
        c = common.shape[0]
        T += c
        t[p] += c
        t[q] += c
        np.add.at(t, common, 1)

    lo, hi = tdist.shard_bounds(n, shard, nshards)   # small-class source rows: a vertex range
    for u in small_rows:
        if lo <= u < hi:
            for v in colp[rpp[u]:rpp[u + 1]]:
                if 1 <= dp[v] <= small_max:
                    edge(u, int(v), colp[rpp[u]:rpp[u + 1]])
    for items, seg_len in ((warp, None), (cta, table_cap)):
        lo, hi = tdist.shard_bounds(len(items), shard, nshards)
        for p, sg, qs in items[lo:hi]:
            keys = colp[rpp[p]:rpp[p + 1]]
            if seg_len:
                keys = keys[sg * seg_len:(sg + 1) * seg_len]
            for q in qs:
                edge(p, q, keys)
    return T, t


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
        # one graph: each rank counts its shard of the work lists, (T, t)
        # combined by one all-reduce (small table segments so that pivots
        # span several CTA items)
        g = gen.rmat(11, 16, seed=3)
        rpp, colp = oracle.orient(g.n, g.row_ptr, g.col)
        T, t = count_share(g.n, rpp, colp, rank, world, table_cap=64)
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
    res = q.get(timeout=300)
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


def test_one_rank_share_is_the_whole_count():
    g = gen.rmat(9, 16, seed=4)
    rpp, colp = oracle.orient(g.n, g.row_ptr, g.col)
    T, t = count_share(g.n, rpp, colp, 0, 1, table_cap=32)
    T1, t1 = oracle.count(g.n, g.row_ptr, g.col)
    assert T == T1 and (t == t1).all()
    # three shards add up to the same
    parts = [count_share(g.n, rpp, colp, k, 3, table_cap=32) for k in range(3)]
    assert sum(p[0] for p in parts) == T1 and (sum(p[1] for p in parts) == t1).all()
