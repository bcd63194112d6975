"""ch_filter_noalloc against ch_filter.

ch_filter_noalloc is for callers that cannot allocate device memory and
cannot hand the library a workspace -- for instance code running inside a
host framework that owns every device allocation, or a path under a fixed
memory budget or a latency budget that cudaMalloc's implicit
synchronisation would break.  Its scratch is a static device array inside
the library, shared by every call and keeping whatever the last call left.

These tests call it through the C ABI twice in a row, on inputs of
different sizes and survivor counts, and require exactly the survivors of
ch_filter (index lists and coordinates bit for bit, the tolerance every
filter test uses), so nothing the first call leaves in the array can leak
into the second.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu


def _filter_both_ways(p):
    d = torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
    n = len(p)
    ws = ch.Workspace(n)
    ext = ch.extremes(d, ws)
    ref_idx, ref_pts, ref_cnt = ch.filter_points(d, ext, ws)
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    pts = torch.full((n, 2), np.nan, dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ch.ch_filter_noalloc(d, ext, idx, pts, cnt)
    torch.cuda.synchronize()
    s_ref, s = int(ref_cnt.item()), int(cnt.item())
    assert s == s_ref
    assert torch.equal(idx[:s], ref_idx[:s])
    assert torch.equal(pts[:s].view(torch.int32), ref_pts[:s].view(torch.int32))
    return s


def test_two_calls_in_a_row_match_ch_filter():
    # first call: every point survives, many tiles; second call: fewer
    # tiles and a handful of survivors, over the same static scratch
    s1 = _filter_both_ways(pointgen.make_points("circle", 1_000_003, seed=31))
    s2 = _filter_both_ways(pointgen.make_points("normal", 300_001, seed=32))
    assert s1 == 1_000_003
    assert 0 < s2 < 1000


def test_largest_size_and_beyond():
    n = 1 << 26
    d = torch.from_numpy(pointgen.make_points("displaced", n, seed=33)).cuda()
    ws = ch.Workspace(n)
    ext = ch.extremes(d, ws)
    ref_idx, _, ref_cnt = ch.filter_points(d, ext, ws, with_points=False)
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ch.ch_filter_noalloc(d, ext, idx, None, cnt)
    torch.cuda.synchronize()
    s = int(cnt.item())
    assert s == int(ref_cnt.item())
    assert torch.equal(idx[:s], ref_idx[:s])
    # one point more is refused on the host, before any device work
    lib = ch.load()
    rc = lib.ch_filter_noalloc(ctypes.c_void_p(d.data_ptr()), n + 1, ctypes.c_void_p(ext.data_ptr()),
                               ctypes.c_void_p(idx.data_ptr()), None, ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == ch.CH_ERR_CAPACITY


def test_second_call_allocates_nothing_on_an_unaligned_view():
    """After the first call (which may load the library's device code and
    looks up the scratch address), a call changes neither the device's free
    memory nor torch's allocations.  The points are a view one point into a
    buffer (8-byte but not 16-byte aligned), so the filter's 8-byte load path
    runs, and its survivors match ch_filter's."""
    p = pointgen.make_points("displaced", 200_001, seed=34)
    big = torch.from_numpy(np.concatenate([np.zeros((1, 2), np.float32), p])).cuda()
    d = big[1:]
    assert d.data_ptr() % 16 == 8
    n = len(p)
    ws = ch.Workspace(n)
    ext = ch.extremes(d, ws)
    ref_idx, ref_pts, ref_cnt = ch.filter_points(d, ext, ws)
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    pts = torch.full((n, 2), np.nan, dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ch.ch_filter_noalloc(d, ext, idx, pts, cnt)
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    ch.ch_filter_noalloc(d, ext, idx, pts, cnt)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == torch0
    s = int(cnt.item())
    assert s == int(ref_cnt.item()) and s > 0
    assert torch.equal(idx[:s], ref_idx[:s])
    assert torch.equal(pts[:s].view(torch.int32), ref_pts[:s].view(torch.int32))


def test_device_error_comes_back_in_the_count():
    """A vertex index beyond n is found on the device; with no workspace to
    query, the count reads NOALLOC_FAILED | CH_ERR_ARG.  The next call,
    over the same scratch, is correct again."""
    p = pointgen.make_points("normal", 50_000, seed=35)
    d = torch.from_numpy(p).cuda()
    bad = torch.tensor([0, 1, 2, 3, 4, 5, 6, 50_000 + 9], dtype=torch.int32, device="cuda")
    idx = torch.empty(len(p), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ch.ch_filter_noalloc(d, bad, idx, None, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) & 0xFFFFFFFF == ch.NOALLOC_FAILED | ch.CH_ERR_ARG
    assert _filter_both_ways(p) > 0
