"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Triangle counts are integers with one correct answer, so every comparison is
bit-exact: the total T, every per-vertex count t(v) and the oriented CSR
itself.  Inputs are seeded synthetic graphs shaped like the benchmark
workloads (Erdos-Renyi, R-MAT with hubs, road-like grids, Barabasi-Albert),
plus closed forms and edge cases."""
from __future__ import annotations

import itertools

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


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_count(ctx, g, per_vertex=True, host=False, validate=False):
    """Build + count through the ABI; returns (T, t or None)."""
    if host:
        o = ctx.build(g.n, g.row_ptr, g.col, validate=validate)
        tot = np.zeros(1, np.int64)
        pv = np.zeros(g.n, np.int64) if per_vertex else None
        ctx.count(o, tot, pv)
        o.free()
        return int(tot[0]), pv
    o = ctx.build(g.n, dev(g.row_ptr), dev(g.col), validate=validate)
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    pv = torch.zeros(g.n, dtype=torch.int64, device="cuda") if per_vertex else None
    ctx.count(o, tot, pv)
    torch.cuda.synchronize()
    o.free()
    return int(tot.item()), (pv.cpu().numpy() if pv is not None else None)


def assert_parity(ctx, g, **kw):
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    Tg, tg = gpu_count(ctx, g, **kw)
    assert Tg == T
    if kw.get("per_vertex", True):
        np.testing.assert_array_equal(tg, t)
    # no device-side check (bounded probes) fired during the count
    assert ctx.check() == 0
    return T


def graph_from_edges(n, edges):
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return gen.from_pairs(n, e[:, 0], e[:, 1])


# ---------------------------------------------------------------- worked example
def test_fig1_example(ctx):
    g = graph_from_edges(7, [(0, 1), (0, 4), (0, 5), (1, 2), (1, 5), (2, 3), (2, 6), (3, 4), (3, 5), (4, 5)])
    T, t = gpu_count(ctx, g)
    assert T == 3
    assert t.tolist() == [2, 1, 0, 1, 2, 3, 0]


def test_oriented_csr_matches_oracle(ctx):
    for g in (gen.rmat(12, 16, seed=1), gen.grid(50, 60, seed=2), gen.er(1024, 8192, seed=3)):
        o = ctx.build(g.n, dev(g.row_ptr), dev(g.col))
        rp, col = o.copy_to_host()
        o.free()
        orp, ocol = oracle.orient(g.n, g.row_ptr, g.col)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(col, ocol)


# ---------------------------------------------------------------- workloads, reduced sizes
@pytest.mark.parametrize("seed", range(10))
def test_er_1024_8192(ctx, seed):
    assert_parity(ctx, gen.er(1024, 8192, seed=seed))


@pytest.mark.parametrize("scale,seed", [(8, 0), (10, 1), (12, 2), (14, 3), (16, 4)])
def test_rmat(ctx, scale, seed):
    assert_parity(ctx, gen.rmat(scale, 16, seed=seed))


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (17, 33), (256, 300)])
def test_grid(ctx, shape):
    assert_parity(ctx, gen.grid(*shape, seed=5))


@pytest.mark.parametrize("n,k", [(100, 2), (2000, 8), (20000, 16)])
def test_ba(ctx, n, k):
    assert_parity(ctx, gen.ba(n, k, seed=n + k))


# every partition class and probe strategy, including forced segmentation of
# pivot lists (table_cap below the max out-degree) and tiny work items
CONFIGS = [
    dict(),
    dict(small_max=-1),
    dict(small_max=64, warp_max=64),
    dict(warp_max=2),
    dict(warp_max=16, table_cap=16, chunk=1),
    dict(probe=2),
    dict(probe=2, table_cap=32, warp_max=8, chunk=3),
    dict(cta_threads=128, chunk=7),
    dict(cta_threads=1024, table_cap=4096, warp_max=1024),
    dict(bitmap_bits=-1),
    dict(direct_span=-1),
    dict(direct_span=-1, bitmap_bits=64, warp_max=4),
    dict(direct_span=40, warp_max=4, chunk=9),
    dict(bitmap_bits=262144, table_cap=64, warp_max=8, chunk=5),
    # the CTA-table kernel with partner lists staged by the copy engine, over
    # every table kind, small tables and tiny work items
    dict(stage=1),
    dict(stage=1, table_cap=64, warp_max=8, chunk=5),
    dict(stage=1, table_cap=16, warp_max=2, chunk=1),
    dict(stage=1, direct_span=-1, bitmap_bits=-1),
    # the degree-ratio switch: balanced edges take the warp merge path
    dict(merge_ratio=200),
    dict(merge_ratio=100, merge_max=16),
    dict(merge_ratio=1000000, merge_max=4096),
    dict(merge_ratio=400, small_max=-1, warp_max=8),
    # threads per row of the thread-merge class
    dict(small_lanes=4),
    dict(small_lanes=32, small_max=64, warp_max=64),
    dict(small_lanes=2, small_max=16, merge_ratio=200),
    dict(small_lanes=8, small_max=32),
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=[str(c) for c in CONFIGS])
def test_partition_configs(B, cfg):
    c = B.Context(0, **cfg)
    for g in (gen.rmat(13, 16, seed=7), gen.ba(3000, 12, seed=1), gen.grid(40, 40, seed=0), gen.er(1024, 8192, seed=9)):
        assert_parity(c, g)
        assert_parity(c, g, per_vertex=False)
    c.close()


def test_merge_class_takes_the_balanced_edges(B):
    """With every non-small edge below the ratio bound, the whole count runs on
    the merge path (and the tables get no work), still bit-exact."""
    g = gen.er(4096, 65536, seed=3)   # d+ mostly 10..30: balanced lists
    c = B.Context(0, merge_ratio=1000000, merge_max=4096)
    c.set_trace(True)
    assert_parity(c, g)
    tr = c.read_trace()
    assert tr["phase_calls"]["count_merge"] >= 1
    c.close()


# ---------------------------------------------------------------- closed forms, edge cases
@pytest.mark.parametrize("D,n", [(255, 256), (255, 70000), (300, 70000), (65535, 70000), (65536, 70000)])
def test_rank_sort_digit_passes(B, D, n):
    """The (degree, id) rank comes from a radix sort over the degree's 8-bit
    digits whose passes above the largest degree's top bit do nothing, so the
    sorted keys end in one buffer or the other by the number of real passes.
    A hub of degree D just below and above 2^8 and 2^16, with n up to 70,000
    (17 id bits), gives one, two and three real passes, with and without
    passes left out.  A wrong buffer scrambles the rank ids of the oriented
    lists, which the table kernels key on: the per-vertex counts of the
    clique's pivots (warp tables by default, CTA tables with warp_max 8) would
    differ from the oracle's."""
    edges = [(0, i) for i in range(1, D + 1)]
    edges += [(i, i + 1) for i in range(1, D)]  # triangles (0, i, i + 1)
    edges += [(i, j) for i in range(1, 41) for j in range(i + 2, 41)]  # with the path, a clique on 1..40
    g = graph_from_edges(n, edges)
    assert int(np.diff(g.row_ptr).max()) == D
    for cfg in ({}, dict(warp_max=8)):
        c = B.Context(0, **cfg)
        assert_parity(c, g)
        c.close()


@pytest.mark.parametrize("n", [3, 4, 33, 200])
def test_complete_graph(ctx, n):
    g = graph_from_edges(n, list(itertools.combinations(range(n), 2)))
    T, t = gpu_count(ctx, g)
    assert T == n * (n - 1) * (n - 2) // 6
    assert (t == (n - 1) * (n - 2) // 2).all()


def test_wheels_and_friendship(ctx):
    for k in (4, 50, 3000, 10000):
        rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
        g = graph_from_edges(k + 1, rim + [(0, 1 + i) for i in range(k)])
        T, t = gpu_count(ctx, g)
        assert T == k and t[0] == k and (t[1:] == 2).all()
    k = 1000
    edges = []
    for i in range(k):
        edges += [(0, 1 + 2 * i), (0, 2 + 2 * i), (1 + 2 * i, 2 + 2 * i)]
    T, t = gpu_count(ctx, graph_from_edges(2 * k + 1, edges))
    assert T == k and t[0] == k and (t[1:] == 1).all()


def test_empty_and_tiny(ctx):
    for n in (1, 2, 5):
        g = gen.from_pairs(n, [], [])
        assert gpu_count(ctx, g) [0] == 0
    g = graph_from_edges(2, [(0, 1)])
    T, t = gpu_count(ctx, g)
    assert T == 0 and t.tolist() == [0, 0]
    g = graph_from_edges(3, [(0, 1), (1, 2), (0, 2)])
    assert gpu_count(ctx, g)[0] == 1


def test_triangle_free(ctx):
    g = graph_from_edges(400, [(i, 200 + j) for i in range(200) for j in range(0, 200, 3)])
    assert gpu_count(ctx, g)[0] == 0
    g = gen.grid(100, 101, seed=0, p_diag=0.0, frac_long=0.0)
    assert gpu_count(ctx, g)[0] == 0


def test_relabel_invariance(ctx):
    g = gen.rmat(12, 16, seed=11)
    T, t = gpu_count(ctx, g)
    perm = np.random.default_rng(0).permutation(g.n).astype(np.int32)
    src = perm[np.repeat(np.arange(g.n), np.diff(g.row_ptr))]
    h = gen.from_pairs(g.n, src, perm[g.col])
    T2, t2 = gpu_count(ctx, h)
    assert T2 == T and (t2[perm] == t).all()


# ---------------------------------------------------------------- input / output placement
def test_host_inputs_and_outputs(ctx):
    g = gen.rmat(11, 16, seed=2)
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    Th, th = gpu_count(ctx, g, host=True)
    assert Th == T and (th == t).all()


def test_pinned_host_inputs(ctx):
    """A pinned host CSR (torch pin_memory: page-locked and mapped for the
    device) is read by the orientation's first pass straight from host
    memory, which leaves the device copy the later passes use.  The oriented
    CSR and the counts equal the oracle's, with host and with device outputs;
    with validation (which reads the input first) the plain upload is taken."""
    for g in (gen.rmat(12, 16, seed=5), gen.grid(60, 70, seed=1), gen.ba(2000, 7, seed=2)):
        rp = torch.from_numpy(g.row_ptr).pin_memory()
        col = torch.from_numpy(g.col).pin_memory()
        orp, ocol = oracle.orient(g.n, g.row_ptr, g.col)
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        for validate in (False, True):
            for host_out in (True, False):
                o = ctx.build(g.n, rp, col, validate=validate)
                hrp, hcol = o.copy_to_host()
                np.testing.assert_array_equal(hrp, orp)
                np.testing.assert_array_equal(hcol, ocol)
                dev_ = "cpu" if host_out else "cuda"
                tot = torch.zeros(1, dtype=torch.int64, device=dev_)
                pv = torch.zeros(g.n, dtype=torch.int64, device=dev_)
                if host_out:
                    tot, pv = tot.pin_memory(), pv.pin_memory()
                ctx.count(o, tot, pv)
                torch.cuda.synchronize()
                o.free()
                assert int(tot[0]) == T
                np.testing.assert_array_equal(pv.cpu().numpy(), t)
    assert ctx.check() == 0


def test_edge_list_input(ctx):
    for g in (gen.rmat(11, 16, seed=4, keep_pairs=True), gen.grid(30, 31, seed=1, keep_pairs=True),
              gen.er(1024, 8192, seed=1, keep_pairs=True)):
        T, t = oracle.count_pairs(g.n, g.src, g.dst)
        # raw pairs hold duplicates, loops (R-MAT) and one direction per pair
        o = ctx.build_edges(g.n, dev(g.src), dev(g.dst))
        rp, col = o.copy_to_host()
        orp, ocol = oracle.orient(g.n, g.row_ptr, g.col)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(col, ocol)
        tot = torch.zeros(1, dtype=torch.int64, device="cuda")
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        ctx.count(o, tot, pv)
        assert int(tot.item()) == T
        np.testing.assert_array_equal(pv.cpu().numpy(), t)
        o.free()
        # host edge list, both directions plus loops
        src = np.concatenate([g.src, g.dst, np.arange(5, dtype=np.int32)])
        dst = np.concatenate([g.dst, g.src, np.arange(5, dtype=np.int32)])
        o = ctx.build_edges(g.n, src, dst)
        tot = np.zeros(1, np.int64)
        ctx.count(o, tot)
        assert int(tot[0]) == T
        o.free()


def test_validation_rejects_bad_csr(B, ctx):
    g = gen.rmat(9, 8, seed=0)
    assert gpu_count(ctx, g, validate=True)[0] == oracle.count(g.n, g.row_ptr, g.col)[0]
    bad = []
    col = g.col.copy(); col[0], col[1] = col[1], col[0]  # unsorted row
    bad.append(col)
    col = g.col.copy(); col[3] = 0 if g.col[3] != 0 else 1  # breaks symmetry / order
    bad.append(col)
    rp = g.row_ptr
    u = int(np.argmax(np.diff(rp) > 0)); col = g.col.copy(); col[rp[u]] = u  # self-loop
    bad.append(col)
    col = g.col.copy(); col[-1] = g.n + 5  # id out of range
    bad.append(col)
    for c in bad:
        with pytest.raises(B.TCError) as ei:
            ctx.build(g.n, dev(g.row_ptr), dev(c), validate=True)
        assert ei.value.status in (B.TC_ERR_INVALID_GRAPH,)
    with pytest.raises(B.TCError):
        ctx.build_edges(4, dev(np.array([0, 1], np.int32)), dev(np.array([1, 9], np.int32)))


def test_many_counts_on_one_handle(ctx):
    g = gen.rmat(12, 16, seed=8)
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    o = ctx.build(g.n, dev(g.row_ptr), dev(g.col))
    streams = [torch.cuda.Stream() for _ in range(3)]
    torch.cuda.synchronize()
    outs = []
    for s in streams:
        tot = torch.zeros(1, dtype=torch.int64, device="cuda")
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        ctx.count(o, tot, pv, stream=s)
        outs.append((tot, pv))
    torch.cuda.synchronize()
    for tot, pv in outs:
        assert int(tot.item()) == T
        np.testing.assert_array_equal(pv.cpu().numpy(), t)
    o.free()


def test_config_out_of_range_is_refused(B):
    for bad in (dict(small_lanes=3), dict(small_lanes=64), dict(table_cap=100), dict(merge_ratio=50)):
        with pytest.raises(B.TCError) as ei:
            B.Context(0, **bad)
        assert ei.value.status == B.TC_ERR_INVALID_ARG, bad
    c = B.Context(0, small_lanes=8)
    got = c.get_config()
    assert got["small_lanes"] == 8
    c.close()
