"""Pins for the CPU oracle (no GPU): each test checks the oracle against
something other than itself -- the paper's worked example, brute force over
vertex triples, dense linear algebra, scipy's sparse products, closed forms
and invariants -- so that a dropped term, a wrong index or a wrong
orientation rule fails at least one of them."""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1804_06926_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    sections, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                sections[cur] = []
                continue
            sections[cur].append([int(x) for x in line.split()])
    return {k: np.array(v, dtype=np.int64) for k, v in sections.items()}


def dense_to_csr(A):
    A = np.asarray(A)
    n = A.shape[0]
    rp = np.zeros(n + 1, np.int64)
    cols = []
    for i in range(n):
        nb = np.nonzero(A[i])[0]
        cols.extend(nb.tolist())
        rp[i + 1] = rp[i] + len(nb)
    return rp, np.array(cols, np.int32)


def csr_to_dense(n, rp, col):
    A = np.zeros((n, n), np.int64)
    for u in range(n):
        A[u, col[rp[u]:rp[u + 1]]] = 1
    return A


def brute_force(n, rp, col):
    """O(n^3) over triples: T and t from the definition."""
    A = csr_to_dense(n, rp, col).astype(bool)
    T = 0
    t = np.zeros(n, np.int64)
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[b, c] and A[a, c]:
            T += 1
            t[[a, b, c]] += 1
    return T, t


def graph_from_edges(n, edges):
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return gen.from_pairs(n, e[:, 0], e[:, 1])


# ---------------------------------------------------------------- worked example
def test_fig1_worked_example_forward():
    g = read_golden("fig1_example.txt")
    A = g["A"]
    assert (A == A.T).all() and A.trace() == 0
    rp, col = dense_to_csr(A)
    T, t = oracle.count(7, rp, col)
    assert T == int(g["T"][0, 0]) == 3
    assert (t == g["t"][0]).all()


def test_fig3_alg3_intermediates():
    """The dense Alg. 3 oracle reproduces Fig. 3's B and C entry by entry."""
    g = read_golden("fig1_example.txt")
    order, L, U, B, C, T = dense.alg3_matrices(g["A"], permute=False)
    assert (L + U == g["A"]).all()
    assert (B == g["B"]).all()
    assert (C == g["C"]).all()
    assert int(C.sum()) == 6 and T == 3
    # the nonzero-count permutation of Alg. 3 step 1 changes B and C but not T
    assert dense.alg3_count(g["A"], permute=True) == 3


# ---------------------------------------------------------------- brute force
def small_graphs():
    out = []
    for s in range(4):
        out.append(("er", gen.er(24 + 4 * s, 60 + 25 * s, seed=s)))
        out.append(("ba", gen.ba(30, 2 + s, seed=s)))
        out.append(("rmat", gen.rmat(5, 4, seed=s)))
    out.append(("grid", gen.grid(5, 6, seed=1, p_diag=0.5, frac_long=0.1)))
    return out


@pytest.mark.parametrize("name,g", small_graphs())
def test_brute_force_triples(name, g):
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    Tb, tb = brute_force(g.n, g.row_ptr, g.col)
    assert T == Tb
    assert (t == tb).all()


@pytest.mark.parametrize("seed", range(5))
def test_trace_a_cubed(seed):
    """T = trace(A^3)/6 and t(v) = (A^3)_vv / 2, dense numpy matmul."""
    for g in (gen.er(150, 900, seed=seed), gen.ba(180, 5, seed=seed), gen.rmat(7, 8, seed=seed)):
        A = csr_to_dense(g.n, g.row_ptr, g.col)
        A3 = A @ A @ A
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        assert 6 * T == int(np.trace(A3))
        assert (2 * t == np.diag(A3)).all()
        assert dense.alg3_count(A) == T


def test_scipy_sparse_medium():
    """Edge-iterator over all directed edges: sum (A^2 o A) = 6T (Sec. 4.2:
    without the filter every triangle is met six times); row sums = 2 t(v)."""
    sp = pytest.importorskip("scipy.sparse")
    for g in (gen.rmat(14, 16, seed=3), gen.er(20000, 120000, seed=1), gen.ba(20000, 8, seed=2),
              gen.grid(120, 130, seed=4)):
        A = sp.csr_matrix((np.ones(g.nnz, np.int64), g.col, g.row_ptr), shape=(g.n, g.n))
        W = (A @ A).multiply(A)
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        assert int(W.sum()) == 6 * T
        assert (np.asarray(W.sum(axis=1)).ravel() == 2 * t).all()


# ---------------------------------------------------------------- closed forms
def comb(n, k):
    from math import comb as c
    return c(n, k)


@pytest.mark.parametrize("n", [3, 4, 5, 10, 31])
def test_complete_graph(n):
    g = graph_from_edges(n, list(itertools.combinations(range(n), 2)))
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    assert T == comb(n, 3)
    assert (t == comb(n - 1, 2)).all()


@pytest.mark.parametrize("k", [3, 4, 5, 9, 40])
def test_wheel(k):
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    spokes = [(0, 1 + i) for i in range(k)]
    g = graph_from_edges(k + 1, rim + spokes)
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    if k == 3:                     # W_3 is K_4
        assert T == 4 and (t == 3).all()
    else:
        assert T == k and t[0] == k and (t[1:] == 2).all()


@pytest.mark.parametrize("k", [1, 2, 7])
def test_friendship(k):
    edges = []
    for i in range(k):
        a, b = 1 + 2 * i, 2 + 2 * i
        edges += [(0, a), (0, b), (a, b)]
    g = graph_from_edges(2 * k + 1, edges)
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    assert T == k and t[0] == k and (t[1:] == 1).all()


def test_triangle_free_families():
    rng = np.random.default_rng(0)
    cases = []
    cases.append(graph_from_edges(12, [(i, 6 + j) for i in range(6) for j in range(6)]))   # K_{6,6}
    parent = [int(rng.integers(0, i)) for i in range(1, 60)]
    cases.append(graph_from_edges(60, [(i + 1, p) for i, p in enumerate(parent)]))         # random tree
    for n in (4, 5, 17):
        cases.append(graph_from_edges(n, [(i, (i + 1) % n) for i in range(n)]))             # C_n
    cases.append(gen.grid(9, 11, seed=0, p_diag=0.0, frac_long=0.0))                       # bipartite lattice
    for g in cases:
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        assert T == 0 and not t.any()


def test_cycle_c3_and_empty():
    g = graph_from_edges(3, [(0, 1), (1, 2), (2, 0)])
    assert oracle.count(3, g.row_ptr, g.col)[0] == 1
    g = gen.from_pairs(5, [], [])
    T, t = oracle.count(5, g.row_ptr, g.col)
    assert T == 0 and t.shape == (5,) and not t.any()


@pytest.mark.parametrize("seed", [0, 1])
def test_grid_diagonals_closed_form(seed):
    """Same-direction diagonals only: each diagonal closes exactly 2 triangles."""
    g = gen.grid(40, 37, seed=seed, p_diag=0.3, frac_long=0.0, keep_pairs=True)
    lattice = 40 * 36 + 39 * 37
    ndiag = g.src.shape[0] - lattice
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    assert ndiag > 0 and T == 2 * ndiag


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(3))
def test_invariants(seed):
    g = gen.rmat(12, 16, seed=seed)
    rpp, colp = oracle.orient(g.n, g.row_ptr, g.col)
    assert colp.shape[0] == g.m                                   # |E+| = m
    deg = np.diff(g.row_ptr)
    u = np.repeat(np.arange(g.n), np.diff(rpp))
    v = colp.astype(np.int64)
    assert ((deg[u] < deg[v]) | ((deg[u] == deg[v]) & (u < v))).all()   # rank(u) < rank(v)
    for a in range(g.n):                                           # rows ascending
        r = colp[rpp[a]:rpp[a + 1]]
        assert (np.diff(r) > 0).all()
    und = set(zip(np.minimum(u, v).tolist(), np.maximum(u, v).tolist()))
    assert len(und) == g.m                                         # each edge kept once
    T, t = oracle.count_oriented(g.n, rpp, colp)
    assert int(t.sum()) == 3 * T
    # strided row subsets partition the count
    assert sum(oracle.count_rows(g.n, rpp, colp, r, g.n, 4) for r in range(4)) == T
    # ... and so do their per-vertex counts
    parts = [oracle.count_rows_pv(g.n, rpp, colp, r, g.n, 3) for r in range(3)]
    assert sum(p[0] for p in parts) == T
    assert (sum(p[1] for p in parts) == t).all()
    # a per-vertex row subset agrees with the definition at its lowest vertex:
    # every triangle of row u (u lowest-ranked) contains u
    Tu, tu = oracle.count_rows_pv(g.n, rpp, colp, 5, 6)
    assert tu[5] == Tu and int(tu.sum()) == 3 * Tu
    # relabelling the vertices permutes t and keeps T
    perm = np.random.default_rng(seed).permutation(g.n).astype(np.int32)
    src = perm[np.repeat(np.arange(g.n), np.diff(g.row_ptr))]
    dst = perm[g.col]
    T2, t2 = oracle.count_pairs(g.n, src, dst)
    assert T2 == T and (t2[perm] == t).all()


def test_vertex_triangles_matches_count():
    g = gen.rmat(11, 16, seed=5)
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    for v in np.random.default_rng(0).choice(g.n, 200, replace=False):
        assert oracle.vertex_triangles(g.n, g.row_ptr, g.col, int(v)) == t[v]


def test_canonicalize_matches_generator_csr():
    """Two independent canonicalisations (oracle's qsort, generator's counting sort)."""
    for g in (gen.rmat(10, 16, seed=2, keep_pairs=True), gen.grid(20, 21, seed=3, keep_pairs=True),
              gen.ba(500, 7, seed=1, keep_pairs=True)):
        rp, col = oracle.canonicalize(g.n, g.src, g.dst)
        assert (rp == g.row_ptr).all() and (col == g.col).all()
    # loops, duplicates and both directions in the raw input
    src = np.array([0, 1, 1, 2, 2, 0, 3, 3, 0], np.int32)
    dst = np.array([1, 0, 2, 1, 0, 2, 3, 3, 1], np.int32)
    rp, col = oracle.canonicalize(4, src, dst)
    assert rp.tolist() == [0, 2, 4, 6, 6]
    assert col.tolist() == [1, 2, 0, 2, 0, 1]
    assert oracle.count_pairs(4, src, dst)[0] == 1


def test_er_expected_triangle_count():
    """Statistical sanity only: G(1024, 8192) has about C(1024,3) p^3 ~ 683 triangles."""
    Ts = [oracle.count(g.n, g.row_ptr, g.col)[0] for g in (gen.er(1024, 8192, seed=s) for s in range(10))]
    p = 8192 / comb(1024, 2)
    expect = comb(1024, 3) * p ** 3
    assert abs(np.mean(Ts) - expect) < 0.1 * expect
