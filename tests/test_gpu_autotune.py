"""Autotuning on the device: every candidate returns the oracle's count and
the chosen configuration is then used for an exact count."""
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


def test_tune_graph_and_batch(B, tmp_path):
    from paper_1804_06926_gb300 import autotune
    tuner = autotune.Autotuner(str(tmp_path / "cache.json"), device_name="test")
    g = gen.rmat(12, 16, seed=4)
    T, t = oracle.count(g.n, g.row_ptr, g.col)
    rp, col = torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()
    res = autotune.tune_graph(g.n, rp, col, tuner=tuner, reps=1)
    # every candidate once, then the greedy merges of those that beat the default
    assert len(res.times_ms) >= len(autotune.CANDIDATES)
    assert [c for c, _ in res.times_ms[:len(autotune.CANDIDATES)]] == autotune.CANDIDATES
    ctx = B.Context(0, **res.best)
    o = ctx.build(g.n, rp, col)
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    ctx.count(o, tot, pv)
    assert int(tot.item()) == T and np.array_equal(pv.cpu().numpy(), t)
    o.free()
    b = gen.ba_batch(16, 100, 1000, 2, 8, seed0=9)
    dev = [torch.from_numpy(x).cuda() for x in (b.vtx_off, b.edge_off, b.row_ptr, b.col)]
    res = autotune.tune_batch(*dev, tuner=tuner, reps=1, candidates=autotune.CANDIDATES[:4])
    # a candidate, or a merge of disjoint candidates
    assert all(any(c.get(k) == v for c in autotune.CANDIDATES[:4]) for k, v in res.best.items())
    # the second call for the same class comes from the cache
    again = autotune.tune_batch(*dev, tuner=tuner, reps=1)
    assert again.best == res.best and again.times_ms == []
