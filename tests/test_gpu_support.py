"""tc_edge_support: per-edge support and the triangle list against the oracle."""
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


def oriented_support(g, rpp, colp):
    """Oracle support of the undirected edge behind every oriented edge."""
    sup = oracle.edge_support(g.n, g.row_ptr, g.col)
    u = np.repeat(np.arange(g.n), np.diff(rpp))
    out = np.empty(colp.shape[0], np.int64)
    for i, (a, b) in enumerate(zip(u.tolist(), colp.tolist())):
        row = g.col[g.row_ptr[a]:g.row_ptr[a + 1]]
        out[i] = sup[g.row_ptr[a] + np.searchsorted(row, b)]
    return out


@pytest.mark.parametrize("g", [gen.rmat(10, 16, seed=2), gen.er(1024, 8192, seed=1), gen.grid(30, 33, seed=1),
                               gen.ba(2000, 6, seed=3)])
def test_support_and_listing(B, g):
    ctx = B.Context(0)
    o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    rpp, colp = o.copy_to_host()
    T, _ = oracle.count(g.n, g.row_ptr, g.col)
    sup = torch.zeros(max(colp.shape[0], 1), dtype=torch.int64, device="cuda")
    tri = torch.zeros(3 * (T + 5), dtype=torch.int32, device="cuda")
    cnt = ctx.edge_support(o, sup, tri)
    assert cnt == T
    np.testing.assert_array_equal(sup.cpu().numpy()[:colp.shape[0]], oriented_support(g, rpp, colp))
    got = tri.cpu().numpy()[:3 * T].reshape(-1, 3)
    want = oracle.list_triangles(g.n, g.row_ptr, g.col)
    assert sorted(map(tuple, got.tolist())) == sorted(map(tuple, want.tolist()))
    # host buffers, a capacity below the count, and count only
    hs = np.zeros(colp.shape[0], np.int64)
    small = np.zeros(3 * max(T // 2, 1), np.int32)
    assert ctx.edge_support(o, hs, small) == T
    np.testing.assert_array_equal(hs, sup.cpu().numpy()[:colp.shape[0]])
    wanted = set(map(tuple, want.tolist()))
    assert all(tuple(t) in wanted for t in small.reshape(-1, 3).tolist()[:min(T, small.shape[0] // 3)])
    assert ctx.edge_support(o) == T
    o.free()


def test_masked_product_matches_dense_alg3(B):
    """c[e] equals Fig. 3's C = A o (LU) at that edge when the rows are ordered
    by decreasing rank (dense Alg. 3 oracle, no nnz permutation of its own)."""
    from oracle import dense
    ctx = B.Context(0)
    for g in (gen.er(300, 2000, seed=4), gen.rmat(8, 8, seed=6), gen.ba(250, 5, seed=1)):
        o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        rpp, colp = o.copy_to_host()
        c = np.zeros(max(colp.shape[0], 1), np.int64)
        T = ctx.masked_product(o, c)
        o.free()
        deg = np.diff(g.row_ptr)
        order = np.lexsort((np.arange(g.n), deg))[::-1]          # decreasing (d, id)
        pos = np.empty(g.n, np.int64)
        pos[order] = np.arange(g.n)
        A = np.zeros((g.n, g.n), np.int64)
        u = np.repeat(np.arange(g.n), deg)
        A[pos[u], pos[g.col]] = 1
        _, _, _, _, Cm, T3 = dense.alg3_matrices(A, permute=False)
        assert T == T3 == oracle.count(g.n, g.row_ptr, g.col)[0]
        uo = np.repeat(np.arange(g.n), np.diff(rpp))
        lo, hi = np.minimum(pos[uo], pos[colp]), np.maximum(pos[uo], pos[colp])
        np.testing.assert_array_equal(c[:colp.shape[0]], Cm[lo, hi])
