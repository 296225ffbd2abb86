"""The TC_DEBUG build of the library (libtc_debug.so, -DTC_DEBUG=1): every
count kernel checks its list, table and cell indexes and the all-zero table
invariant at the start of each work item, raises a bit of the device check
word on a violation and skips the access.  compute-sanitizer is closed on this
pool, so these checks stand in for it: the small parity cases run under the
debug build, in a process of their own, in every partition class and probe
mode, and must be bit-exact with no check raised."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import itertools, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle
from paper_1804_06926_gb300 import binding, gen
lib = binding.load()
assert binding.library_path().endswith('libtc_debug.so'), binding.library_path()

def graphs():
    yield 'er', gen.er(1024, 8192, seed=0)
    yield 'rmat12', gen.rmat(12, 16, seed=0)
    yield 'grid', gen.grid(64, 64, seed=0)
    yield 'ba', gen.ba(3000, 12, seed=1)
    k = 300
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)] + [(0, 1 + i) for i in range(k)]
    e = np.array(rim, np.int32)
    yield 'wheel', gen.from_pairs(k + 1, e[:, 0], e[:, 1])
    kn = np.array(list(itertools.combinations(range(60), 2)), np.int32)
    yield 'K60', gen.from_pairs(60, kn[:, 0], kn[:, 1])

cfgs = [dict(), dict(stage=1), dict(stage=1, table_cap=64, warp_max=8, chunk=5),
        dict(direct_span=-1), dict(direct_span=-1, bitmap_bits=-1), dict(probe=2),
        dict(merge_ratio=300), dict(small_max=-1, warp_max=2)]
for cfg in cfgs:
    ctx = binding.Context(0, **cfg)
    for name, g in graphs():
        T, t = oracle.count(g.n, g.row_ptr, g.col)
        o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        tot = torch.zeros(1, dtype=torch.int64, device='cuda')
        pv = torch.zeros(g.n, dtype=torch.int64, device='cuda')
        ctx.count(o, tot, pv)
        bits = ctx.check()
        o.free()
        assert bits == 0, (cfg, name, bits)
        assert int(tot.item()) == T, (cfg, name)
        assert np.array_equal(pv.cpu().numpy(), t), (cfg, name)
    ctx.close()
print('debug build ok')
"""


def test_debug_build_parity_without_a_check_raised():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, TC_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], env=env, capture_output=True,
                       text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout
