"""Pins for the edge-support and listing oracle (no GPU): scipy's A^2 o A and
brute force over triples."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1804_06926_gb300 import gen


def brute_triangles(g):
    A = np.zeros((g.n, g.n), bool)
    for u in range(g.n):
        A[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = True
    return {t for t in itertools.combinations(range(g.n), 3) if A[t[0], t[1]] and A[t[1], t[2]] and A[t[0], t[2]]}


@pytest.mark.parametrize("g", [gen.er(40, 200, seed=1), gen.ba(50, 4, seed=2), gen.rmat(5, 6, seed=3)])
def test_listing_matches_brute_force(g):
    tri = oracle.list_triangles(g.n, g.row_ptr, g.col)
    assert {tuple(sorted(t)) for t in tri.tolist()} == brute_triangles(g)
    assert len({tuple(sorted(t)) for t in tri.tolist()}) == len(tri)  # each once


def test_support_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    for g in (gen.rmat(12, 16, seed=4), gen.ba(4000, 7, seed=1), gen.grid(40, 45, seed=2)):
        A = sp.csr_matrix((np.ones(g.nnz, np.int64), g.col, g.row_ptr), shape=(g.n, g.n))
        W = (A @ A).multiply(A).tocsr()
        W.sort_indices()
        sup = oracle.edge_support(g.n, g.row_ptr, g.col)
        ref = np.zeros(g.nnz, np.int64)
        for u in range(g.n):  # W keeps only nonzero support entries; place them by column
            cols = W.indices[W.indptr[u]:W.indptr[u + 1]]
            vals = W.data[W.indptr[u]:W.indptr[u + 1]]
            pos = g.row_ptr[u] + np.searchsorted(g.col[g.row_ptr[u]:g.row_ptr[u + 1]], cols)
            ref[pos] = vals
        np.testing.assert_array_equal(sup, ref)
        T, _ = oracle.count(g.n, g.row_ptr, g.col)
        assert int(sup.sum()) == 6 * T  # each triangle: 3 edges, both directions
