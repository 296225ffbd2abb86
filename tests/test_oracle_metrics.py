"""Pins for the metric oracle (no GPU): networkx and closed forms."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1804_06926_gb300 import gen

nx = pytest.importorskip("networkx")


def to_nx(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    G.add_edges_from(zip(u.tolist(), g.col.tolist()))
    return G


@pytest.mark.parametrize("g", [gen.er(300, 2000, seed=1), gen.ba(400, 6, seed=2), gen.rmat(9, 8, seed=3),
                               gen.grid(20, 20, seed=0)])
def test_against_networkx(g):
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    G = to_nx(g)
    c = metrics.local_clustering(g.row_ptr, t)
    ref = nx.clustering(G)
    np.testing.assert_allclose(c, [ref[v] for v in range(g.n)], rtol=0, atol=1e-15)
    assert abs(metrics.transitivity(T, g.row_ptr) - nx.transitivity(G)) <= 1e-15
    assert int(metrics.wedges(g.row_ptr).sum()) == sum(d * (d - 1) // 2 for _, d in G.degree())


def test_closed_forms():
    n = 9
    e = np.array(list(itertools.combinations(range(n), 2)), np.int32)
    g = gen.from_pairs(n, e[:, 0], e[:, 1])
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    assert (metrics.local_clustering(g.row_ptr, t) == 1.0).all() and metrics.transitivity(T, g.row_ptr) == 1.0
    star = gen.from_pairs(7, np.zeros(6, np.int32), np.arange(1, 7, dtype=np.int32))
    T, t = oracle.count(star.n, star.row_ptr, star.col)
    assert not metrics.local_clustering(star.row_ptr, t).any() and metrics.transitivity(T, star.row_ptr) == 0.0
    k = 8
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)] + [(0, 1 + i) for i in range(k)]
    e = np.array(rim, np.int32)
    w = gen.from_pairs(k + 1, e[:, 0], e[:, 1])
    T, t = oracle.count(w.n, w.row_ptr, w.col)
    c = metrics.local_clustering(w.row_ptr, t)
    assert c[0] == 2.0 / (k - 1) and (c[1:] == 2.0 / 3.0).all()
