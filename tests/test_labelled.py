"""Labelled-triangle counts (Alg. 1): oracle pinned to brute force on CPU,
GPU subgraph-matching path against the oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1804_06926_gb300 import gen


def brute(g, lab, query):
    A = np.zeros((g.n, g.n), bool)
    for u in range(g.n):
        A[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = True
    q = sorted(query)
    return sum(1 for t in itertools.combinations(range(g.n), 3)
               if A[t[0], t[1]] and A[t[1], t[2]] and A[t[0], t[2]] and sorted(lab[list(t)]) == q)


QUERIES = [(0, 1, 2), (0, 0, 1), (2, 1, 1), (1, 1, 1), (0, 0, 0), (3, 3, 3), (0, 2, 5)]


def test_oracle_labelled_matches_brute_force():
    rng = np.random.default_rng(0)
    for g in (gen.er(40, 250, seed=1), gen.ba(45, 5, seed=2)):
        lab = rng.integers(0, 3, g.n).astype(np.int32)
        for q in QUERIES:
            assert oracle.count_labelled(g.n, g.row_ptr, g.col, lab, q) == brute(g, lab, q)
    # one label everywhere: the plain count
    g = gen.rmat(9, 8, seed=4)
    assert oracle.count_labelled(g.n, g.row_ptr, g.col, np.zeros(g.n, np.int32), (0, 0, 0)) == \
        oracle.count(g.n, g.row_ptr, g.col, per_vertex=False)[0]


@pytest.mark.gpu
def test_gpu_labelled_counts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06926_gb300 import binding
    ctx = binding.Context(0)
    rng = np.random.default_rng(1)
    for g in (gen.rmat(12, 16, seed=3), gen.er(1024, 8192, seed=2), gen.ba(5000, 8, seed=1)):
        rp, col = torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()
        for k in (1, 3, 4):
            lab = rng.integers(0, k, g.n).astype(np.int32)
            dl = torch.from_numpy(lab).cuda()
            for q in QUERIES:
                assert ctx.count_labelled(g.n, rp, col, dl, q) == oracle.count_labelled(g.n, g.row_ptr, g.col, lab, q)
