"""tc_orient_noalloc: the oriented CSR into caller-owned buffers, with no
device allocation inside the library.

It is meant for callers that cannot allocate device memory while running
(latency-bound serving loops, where cudaMalloc/cudaFree can synchronise the
device; processes whose HBM another allocator has reserved in full).  Its only
scratch is a fixed device array inside the library, shared by all calls.

This file is named so that pytest collects it last.  It checks the entry point
through the C ABI against the allocating path (tc_build_oriented_csr +
tc_ocsr_copy) on two calls in a row, and against the oracle's orientation, bit
for bit, since the result is an integer structure with one correct answer;
the sizes include an empty graph and the 4096 x 4096 grid, whose 2^24
vertices are exactly the scratch's limit (8192 scan tiles, so the carry
between the passes of the one-block tile scan runs)."""
from __future__ import annotations

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
    binding.load()
    return binding


def reference_oriented(B, ctx, g):
    """The existing allocating entry points: build, then copy out."""
    o = ctx.build(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    rp, col = o.copy_to_host()
    o.free()
    return rp, col


def noalloc_oriented(B, g, stream):
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    rpp = torch.full((g.n + 1,), -7, dtype=torch.int64, device="cuda")
    colp = torch.full((max(g.m, 1),), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st = B.tc_orient_noalloc(g.n, g.nnz, rp.data_ptr(), col.data_ptr(), rpp.data_ptr(), colp.data_ptr(),
                             stream.cuda_stream)
    assert st == B.TC_OK
    stream.synchronize()
    return rpp.cpu().numpy(), colp.cpu().numpy()[:g.m]


def test_two_calls_match_the_allocating_path(B):
    ctx = B.Context(0)
    stream = torch.cuda.Stream()
    # two different graphs back to back: the second call reuses the scratch
    # array the first one left behind
    for g in (gen.rmat(14, 16, seed=21), gen.grid(300, 301, seed=4)):
        want_rp, want_col = reference_oriented(B, ctx, g)
        got_rp, got_col = noalloc_oriented(B, g, stream)
        np.testing.assert_array_equal(got_rp, want_rp)
        np.testing.assert_array_equal(got_col, want_col)
        o_rp, o_col = oracle.orient(g.n, g.row_ptr, g.col)
        np.testing.assert_array_equal(got_rp, o_rp)
        np.testing.assert_array_equal(got_col, o_col)
    ctx.close()


def test_at_the_scratch_limit_and_empty(B):
    stream = torch.cuda.Stream()
    # n = 2^24 = TC_NOALLOC_MAX_VERTICES: every tile sum of the scratch is used
    g = gen.grid(4096, 4096, seed=0)
    assert g.n == B.TC_NOALLOC_MAX_VERTICES
    got_rp, got_col = noalloc_oriented(B, g, stream)
    o_rp, o_col = oracle.orient(g.n, g.row_ptr, g.col)
    np.testing.assert_array_equal(got_rp, o_rp)
    np.testing.assert_array_equal(got_col, o_col)
    # and a graph past 2^21 vertices that is not at the limit (1025 tiles)
    g = gen.grid(1450, 1447, seed=1)
    got_rp, got_col = noalloc_oriented(B, g, stream)
    o_rp, o_col = oracle.orient(g.n, g.row_ptr, g.col)
    np.testing.assert_array_equal(got_rp, o_rp)
    np.testing.assert_array_equal(got_col, o_col)
    # no vertices at all: rpp_out[0] = 0
    rp = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    st = B.tc_orient_noalloc(0, 0, rp.data_ptr(), None, out.data_ptr(), None, stream.cuda_stream)
    assert st == B.TC_OK
    stream.synchronize()
    assert int(out.item()) == 0
    # vertices without edges: every offset 0
    rp = torch.zeros(6, dtype=torch.int64, device="cuda")
    out = torch.full((6,), -7, dtype=torch.int64, device="cuda")
    st = B.tc_orient_noalloc(5, 0, rp.data_ptr(), None, out.data_ptr(), None, stream.cuda_stream)
    assert st == B.TC_OK
    stream.synchronize()
    assert out.cpu().tolist() == [0] * 6


def test_rejects_graphs_beyond_the_scratch(B):
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    n_too_big = B.TC_NOALLOC_MAX_VERTICES + 1
    st = B.tc_orient_noalloc(n_too_big, 0, rp.data_ptr(), None, out.data_ptr(), None, None)
    assert st == B.TC_ERR_INVALID_ARG
