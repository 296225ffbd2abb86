"""tc_count_shard: the shards of one oriented CSR add up to tc_count."""
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


@pytest.mark.parametrize("nshards", [1, 2, 3, 8])
def test_shards_sum_to_the_count(B, nshards):
    from paper_1804_06926_gb300 import dist as tdist
    ctx = B.Context(0, warp_max=32)
    for g in (gen.rmat(14, 16, seed=2), gen.grid(200, 210, seed=1), gen.ba(5000, 9, seed=4)):
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        tot = torch.zeros(1, dtype=torch.int64, device="cuda")
        pv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        tdist.count_sharded_one_device(ctx, o, nshards, tot, pv)
        torch.cuda.synchronize()
        assert int(tot.item()) == T
        np.testing.assert_array_equal(pv.cpu().numpy(), t)
        if nshards > 1:  # a single shard is a strict part of the work
            part = torch.zeros(1, dtype=torch.int64, device="cuda")
            ctx.count_shard(o, 0, nshards, part)
            torch.cuda.synchronize()
            assert 0 <= int(part.item()) <= T
        o.free()


def test_shard_arguments_are_checked(B):
    ctx = B.Context(0)
    g = gen.rmat(8, 8, seed=1)
    o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    for sh, ns in ((0, 0), (2, 2), (-1, 3)):
        with pytest.raises(B.TCError):
            ctx.count_shard(o, sh, ns, tot)
    o.free()
