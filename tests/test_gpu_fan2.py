"""The hull step's second fan level (sets whose first level leaves at least
2^19 points, 2^16 here through its tuning knob): the survivors of the first level are tested again against a
fan with eight times as many bins whose vertices are the farthest
survivors of their sub-bins, and only the rest is sorted.  Hulls through
ch_hull, element by element against the oracle: the unit circle (where the
first level leaves about a sixth of the points), an 8-byte-aligned view,
every point twice (ties between equal points go to the lowest index),
scales where the binary32 signs overflow or underflow (the exact tiers
decide), and a set where the level does not run."""
import numpy as np
import pytest
import torch

import oracle
import oracle_par
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu

N = (1 << 22) + 13
MIN_LOG2 = 16     # the second level's threshold in these tests (built-in: 2^19 first-level survivors)
MIN_S = 1 << MIN_LOG2


@pytest.fixture(autouse=True)
def low_threshold():
    ch.ch_tune_set("fan2_min_log2", MIN_LOG2)
    try:
        yield
    finally:
        ch.ch_tune_set("fan2_min_log2", 0)


def run(p, offset=False):
    """(hull, counts) of ch_hull on a fresh workspace; offset: the points
    start 8 bytes past a 16-byte boundary."""
    if offset:
        big = torch.from_numpy(np.concatenate([np.zeros((1, 2), np.float32), p])).cuda()
        d = big[1:]
        assert d.data_ptr() % 16 == 8
    else:
        d = torch.from_numpy(p).cuda()
    ws = ch.Workspace(len(p))
    hidx, hcnt = ch.convex_hull(d, ws)
    ws.check()
    c = ch.ch_hull_counts(ws.buf, len(p))
    h = hidx[: int(hcnt.item())].cpu().numpy().view(np.uint32)
    del d, ws, hidx
    torch.cuda.synchronize()
    return h, c


def want_hull(p):
    return oracle_par.hull(p, oracle_par.filter_points(p, oracle.extremes(p)))


@pytest.mark.parametrize("offset", [False, True])
def test_circle(offset):
    p = pointgen.make_points("circle", N, seed=21)
    h, (s_oct, t, spec, t1) = run(p, offset)
    assert spec == 0 and t1 >= MIN_S, (t1, t)
    assert t < t1, (t1, t)   # the second level drops survivors of the first
    assert np.array_equal(h, want_hull(p))


def test_every_point_twice():
    base = pointgen.make_points("circle", N // 2, seed=22)
    rng = np.random.default_rng(22)
    p = np.concatenate([base, base])[rng.permutation(2 * len(base))]
    h, (_, t, _, t1) = run(p)
    assert t1 >= MIN_S and t < t1
    assert np.array_equal(h, want_hull(p))


@pytest.mark.parametrize("scale", [2.0 ** 100, 2.0 ** -100])
def test_scaled_circle(scale):
    # a power-of-two scale keeps the binary32 points' structure; the
    # products of the binary32 signs overflow (underflow) and the exact
    # tiers decide
    p = (pointgen.make_points("circle", N, seed=23).astype(np.float64) * scale).astype(np.float32)
    h, (_, t, _, t1) = run(p)
    assert np.array_equal(h, want_hull(p))


def test_level_off_when_few_survive():
    p = pointgen.make_points("displaced", N, seed=24)
    h, (_, t, _, t1) = run(p)
    assert t1 == t < MIN_S
    assert np.array_equal(h, want_hull(p))


def test_workspace_reuse_after_the_second_level():
    # a call with the second level, then one without, on the same workspace
    p1 = pointgen.make_points("circle", N, seed=25)
    p2 = pointgen.make_points("normal", N, seed=26)
    ws = ch.Workspace(N)
    for p in (p1, p2, p1):
        d = torch.from_numpy(p).cuda()
        hidx, hcnt = ch.convex_hull(d, ws)
        ws.check()
        assert np.array_equal(hidx[: int(hcnt.item())].cpu().numpy().view(np.uint32), want_hull(p))
