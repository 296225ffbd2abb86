"""tc_count_graph: the one-call path, whose small graphs take one fused kernel.

Every result is compared bit for bit with the CPU oracle (T and every t(v)),
and with build + count on the same graph.  The trace's launch count shows
which path ran: one launch for a graph that fits one CTA's shared memory, the
general path otherwise (over the vertex limit, over the shared-memory limit,
or with TC_VALIDATE)."""
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


def fused_words(n, m):
    """Shared-memory words of the fused kernel (row offsets, counts, oriented
    offsets, keep bits and their prefix, N+, scan)."""
    w = (2 * m + 31) // 32
    return (n + 1) + n + (n + 1) + 2 * w + m + 33


def fits(g):
    return g.n <= 8192 and 4 * fused_words(g.n, g.nnz // 2) <= 224 * 1024


def one_call(ctx, g, host_in=False, host_out=False, per_vertex=True, validate=False):
    """(T, t, launches) through tc_count_graph."""
    rp, col = (g.row_ptr, g.col) if host_in else (dev(g.row_ptr), dev(g.col))
    if host_out:
        tot = np.full(1, -7, np.int64)
        pv = np.full(g.n, -7, np.int64) if per_vertex else None
    else:
        tot = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        pv = torch.full((g.n,), -7, dtype=torch.int64, device="cuda") if per_vertex else None
    ctx.read_trace()
    ctx.set_trace(True)
    ctx.count_graph(g.n, rp, col, tot, pv, validate=validate)
    torch.cuda.synchronize()
    ctx.set_trace(False)
    launches = ctx.read_trace()["launches"]
    if not host_out:
        tot = tot.cpu().numpy()
        pv = pv.cpu().numpy() if pv is not None else None
    return int(tot[0]), pv, launches


def check(ctx, g, **kw):
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    Tg, tg, launches = one_call(ctx, g, **kw)
    assert Tg == T
    if kw.get("per_vertex", True):
        np.testing.assert_array_equal(tg, t)
    return launches


def complete(n):
    e = np.array(list(itertools.combinations(range(n), 2)), np.int32).reshape(-1, 2)
    return gen.from_pairs(n, e[:, 0], e[:, 1])


def wheel(k):
    src = [0] * k + list(range(1, k + 1))
    dst = list(range(1, k + 1)) + [1 + (i % k) for i in range(1, k + 1)]
    return gen.from_pairs(k + 1, src, dst)


@pytest.mark.parametrize("seed", range(5))
def test_er_fused(ctx, seed):
    g = gen.er(1024, 8192, seed=seed)
    assert fits(g)
    assert check(ctx, g) == 1


@pytest.mark.parametrize("scale", [6, 8, 10, 11])
def test_rmat_fused(ctx, scale):
    g = gen.rmat(scale, 16, seed=scale)
    assert fits(g)
    assert check(ctx, g) == 1


@pytest.mark.parametrize("seed", range(3))
def test_ba_and_grid_fused(ctx, seed):
    for g in (gen.ba(3000, 6, seed=seed), gen.grid(60, 70, seed=seed)):
        assert fits(g)
        assert check(ctx, g) == 1


def test_closed_forms(ctx):
    from math import comb
    g = complete(120)
    T, _, launches = one_call(ctx, g)
    assert T == comb(120, 3) and launches == 1
    for k in (3, 4, 5, 300):
        T, t, _ = one_call(ctx, wheel(k))
        assert T == (4 if k == 3 else k)
        assert int(t.sum()) == 3 * T
    star = gen.from_pairs(50, [0] * 49, list(range(1, 50)))
    T, t, _ = one_call(ctx, star)
    assert T == 0 and not t.any()


def test_degenerate(ctx):
    for n in (0, 1, 2, 10):
        g = gen.from_pairs(n, [], [])
        T, t, launches = one_call(ctx, g)
        assert T == 0 and launches == 1
        assert t.shape == (n,) and not t.any()
    g = gen.from_pairs(2, [0], [1])
    T, t, _ = one_call(ctx, g)
    assert T == 0 and list(t) == [0, 0]
    g = gen.from_pairs(3, [0, 1, 2], [1, 2, 0])
    T, t, _ = one_call(ctx, g)
    assert T == 1 and list(t) == [1, 1, 1]


@pytest.mark.parametrize("host_in,host_out", [(True, False), (False, True), (True, True)])
def test_host_buffers(ctx, host_in, host_out):
    g = gen.rmat(9, 16, seed=3)
    assert check(ctx, g, host_in=host_in, host_out=host_out) == 1


def test_without_per_vertex(ctx):
    g = gen.er(1024, 8192, seed=11)
    assert check(ctx, g, per_vertex=False) == 1


def test_limits_fall_back(ctx):
    # just over the vertex limit, and over the shared-memory limit: general path
    for g in (gen.er(8193, 20000, seed=1), gen.rmat(13, 16, seed=1)):
        assert not fits(g)
        assert check(ctx, g) > 1
    # the largest vertex count the kernel takes
    g = gen.er(8192, 12000, seed=2)
    assert fits(g)
    assert check(ctx, g) == 1
    # TC_VALIDATE takes the general path
    assert check(ctx, gen.er(1024, 8192, seed=3), validate=True) > 1


def test_same_as_build_and_count(ctx):
    g = gen.rmat(11, 16, seed=5)
    o = ctx.build(g.n, dev(g.row_ptr), dev(g.col))
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    ctx.count(o, tot, pv)
    torch.cuda.synchronize()
    o.free()
    T, t, _ = one_call(ctx, g)
    assert T == int(tot.item())
    np.testing.assert_array_equal(t, pv.cpu().numpy())
    # repeated calls on the same outputs overwrite them
    T2, t2, _ = one_call(ctx, g)
    assert T2 == T
    np.testing.assert_array_equal(t2, t)
