"""tc_clustering against the metric oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1804_06926_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06926_gb300 import binding
    return binding


def test_clustering_and_transitivity(B):
    ctx = B.Context(0)
    for g in (gen.rmat(13, 16, seed=1), gen.er(1024, 8192, seed=0), gen.grid(64, 70, seed=2), gen.ba(3000, 5, seed=9),
              gen.from_pairs(4, [], [])):
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        tot = torch.zeros(1, dtype=torch.int64, device="cuda")
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        ctx.count(o, tot, pv)
        local = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        tr, W = ctx.clustering(o, tot, pv, local)
        np.testing.assert_array_equal(local.cpu().numpy(), metrics.local_clustering(g.row_ptr, t))
        assert tr == metrics.transitivity(T, g.row_ptr)
        assert W == int(metrics.wedges(g.row_ptr).sum())
        host_local = np.zeros(g.n, np.float64)
        ctx.clustering(o, tot, pv, host_local)
        np.testing.assert_array_equal(host_local, metrics.local_clustering(g.row_ptr, t))
        o.free()
