"""The speculative single sweep (sets of at least 2^22 points, two-pass
schedule): a sample octagon P0 is built first, the extremes sweep writes
the points it cannot prove strictly inside P0 as candidates, and when its
last block proves P0 inside the final octagon the filter tests only the
candidates.  Through ch_extremes_filter (vertices and survivor lists) and
ch_hull (hulls), element by element against the oracle, both when the
speculation serves the filter and when it falls back: a probe of evenly
spaced points that predicts an overflow (the unit circle: nothing is
inside), a candidate segment that overflows although the probe passed, a
sample vertex outside the final octagon (planted), and the single-pass
schedule."""
import numpy as np
import pytest
import torch

import oracle
import oracle_par
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu

N = (1 << 22) + 13   # odd: the last point is handled apart from the point pairs


def run(p, offset=False):
    """(ext8, survivors, survivor coordinates, hull, speculation used) from
    ch_extremes_filter and ch_hull on one workspace; offset: the points
    start 8 bytes past a 16-byte boundary."""
    if offset:
        big = torch.from_numpy(np.concatenate([np.zeros((1, 2), np.float32), p])).cuda()
        d = big[1:]
        assert d.data_ptr() % 16 == 8
    else:
        d = torch.from_numpy(p).cuda()
    ws = ch.Workspace(len(p))
    e, idx, sp, cnt = ch.extremes_and_filter(d, ws)
    ws.check()
    s = int(cnt.item())
    hidx, hcnt = ch.convex_hull(d, ws)
    ws.check()
    spec = ch.ch_hull_counts(ws.buf, len(p))[2]
    out = (e.cpu().numpy().view(np.uint32), idx[:s].cpu().numpy().view(np.uint32), sp[:s].cpu().numpy(),
           hidx[: int(hcnt.item())].cpu().numpy().view(np.uint32), spec)
    del d, ws, idx, sp, hidx
    torch.cuda.synchronize()
    return out


def check(p, got):
    e, s, spts, h, _ = got
    oe = oracle.extremes(p)
    assert np.array_equal(e, oe), (e, oe)
    want = oracle_par.filter_points(p, oe)
    assert np.array_equal(s, want), (len(s), len(want))
    assert np.array_equal(spts.view(np.uint32), p[want].view(np.uint32))
    assert np.array_equal(h, oracle_par.hull(p, want))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_normal_served_by_candidates(seed):
    p = pointgen.make_points("normal", N, seed=seed)
    got = run(p)
    check(p, got)
    assert got[4] == 1


def test_normal_unaligned_view():
    # the set of the first case, read through 8-byte loads: the same outcome
    p = pointgen.make_points("normal", N, seed=1)
    got = run(p, offset=True)
    check(p, got)
    assert got[4] == 1


def test_survivors_in_first_middle_and_last_segment():
    # new extremes at the first, the middle and the last index: survivors in
    # the first, a middle and the last candidate segment (the last index is
    # the odd point after the point pairs, written by the last sweep block),
    # in index order
    p = pointgen.make_points("normal", N, seed=5)
    p[0] = (-6.5, 0.3)
    p[N // 2] = (0.2, 6.8)
    p[N - 1] = (7.0, 0.5)
    got = run(p)
    check(p, got)
    assert got[4] == 1
    assert {0, N // 2, N - 1} <= set(got[1].tolist())


def test_normal_sample_octagon_outside_falls_back():
    # for this set a vertex of the sample octagon lies outside the final
    # octagon (checked on the host with binary64 signs: about one set in
    # twelve at this size), so the filter's two passes run
    p = pointgen.make_points("normal", N, seed=4)
    got = run(p)
    check(p, got)
    assert got[4] == 0


def test_circle_falls_back():
    # no point is inside any octagon of circle points: the probe sees them
    # all outside the sample's region and the sweep does not speculate
    p = pointgen.make_points("circle", N, seed=6)
    got = run(p)
    check(p, got)
    assert got[4] == 0


def test_segment_overflow_after_the_probe_passed():
    # normal points at the probe's indices (k * (N // 1024)) and in the 32
    # sample runs, every other point on a circle of radius 6, outside the
    # sample's region (about 0.9 of the sample extremes, near 4): the probe
    # finds nothing outside, the sweep's candidate segments overflow
    p = pointgen.make_points("normal", N, seed=10)
    keep = np.zeros(N, bool)
    keep[np.arange(1024) * (N // 1024)] = True
    for b in range(32):
        s0 = (N - 2048) * b // 31
        keep[s0:s0 + 2048] = True
    ring = pointgen.make_points("circle", N, seed=11).astype(np.float64) * 6.0
    p[~keep] = ring[~keep].astype(np.float32)
    got = run(p)
    check(p, got)
    assert got[4] == 0


def _planted(seed, r_extra):
    """Normal(0,1) points with the final octagon's vertices at radius 100
    (between the sample runs), the sample octagon's at radius 50 (at the
    starts of sample runs 0..7), and one more sample point at radius
    r_extra on the bisector of the edge R -> TR (start of run 8): an
    extreme in no direction for r_extra < 108.2.  With the sample box's
    centre c = ((0.924 r_extra - 50) / 2, 0), that point moved to 0.9 of the
    way from c lies 0.9427 r_extra - 2.31 from the origin along the
    bisector, outside the final octagon (inradius 100 cos(pi/8) = 92.39)
    for r_extra > 100.5."""
    p = pointgen.make_points("normal", N, seed=seed)
    run = lambda b: (N - 2048) * b // 31   # first index of sample run b
    for k in range(8):
        a = k * np.pi / 4
        p[run(k)] = (50 * np.cos(a), 50 * np.sin(a))
        p[(run(k) + run(k + 1)) // 2] = (100 * np.cos(a), 100 * np.sin(a))
    p[run(8)] = (r_extra * np.cos(np.pi / 8), r_extra * np.sin(np.pi / 8))
    return p


def test_sample_vertex_outside_the_octagon_falls_back():
    # the sample octagon reaches beyond the final one: its exact check fails
    # (there are no candidates to overflow: the cloud lies well inside it)
    p = _planted(7, 107.0)
    got = run(p)
    check(p, got)
    assert got[4] == 0


def test_sample_octagon_inside_is_used():
    p = _planted(7, 95.0)
    got = run(p)
    check(p, got)
    assert got[4] == 1


def test_single_pass_schedule_does_not_speculate():
    p = pointgen.make_points("normal", N, seed=8)
    ch.ch_filter_variant(1)
    try:
        got = run(p)
    finally:
        ch.ch_filter_variant(0)
    check(p, got)
    assert got[4] == 0


@pytest.mark.parametrize("n", [(1 << 22) - 1, 100_003])
def test_below_the_size_threshold(n):
    p = pointgen.make_points("normal", n, seed=9)
    got = run(p)
    check(p, got)
    assert got[4] == 0
