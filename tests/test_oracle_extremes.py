"""Pins for the oracle's polygon vertices (Sec. 3.1, findingPolygon).

Brute force in numpy binary32 (first occurrence = lowest index), exhaustive
tie cases, the Manhattan-distance definition of the corner points on inputs
where every key is exact, and non-finite rejection.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import pointgen


def brute_extremes(p):
    p = np.asarray(p, np.float32)
    x, y = p[:, 0], p[:, 1]
    s = (x + y).astype(np.float32)
    d = (x - y).astype(np.float32)
    return np.array([
        np.argmax(x), np.argmax(s), np.argmax(y), np.argmin(d),
        np.argmin(x), np.argmin(s), np.argmin(y), np.argmax(d),
    ], dtype=np.uint32)


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 4099])
def test_matches_brute_force(dist, n):
    p = pointgen.make_points(dist, n, seed=n + 7)
    assert np.array_equal(oracle.extremes(p), brute_extremes(p))


def test_all_equal_points_give_index_zero():
    p = np.full((50, 2), 3.25, np.float32)
    assert np.array_equal(oracle.extremes(p), np.zeros(8, np.uint32))


def test_ties_take_lowest_index():
    # a 3x3 grid listed twice: every extreme key is tied many times
    g = np.array([(x, y) for x in (-1, 0, 1) for y in (-1, 0, 1)], np.float32)
    p = np.concatenate([g[::-1], g])
    e = oracle.extremes(p)
    assert np.array_equal(e, brute_extremes(p))
    # R = first point with x == 1 in p, etc.
    assert p[e[0], 0] == 1 and np.all(p[: e[0], 0] < 1)
    assert p[e[4], 0] == -1 and np.all(p[: e[4], 0] > -1)


def test_signed_zero_ties():
    p = np.array([(0.0, 1.0), (-0.0, 1.0), (0.0, -1.0), (-0.0, -1.0)], np.float32)
    assert np.array_equal(oracle.extremes(p), brute_extremes(p))


def test_corners_minimise_manhattan_distance_to_box_corners():
    """Sec. 3.1: a corner point is the point closest, in Manhattan distance,
    to a corner of the bounding box.  With small-integer coordinates every
    sum is exact, so the closest point (lowest index on ties) must be the
    oracle's TR / TL / BL / BR."""
    rng = np.random.default_rng(3)
    for trial in range(40):
        p = rng.integers(-20, 21, size=(int(rng.integers(1, 60)), 2)).astype(np.float32)
        e = oracle.extremes(p)
        q = [(Fraction(int(a)), Fraction(int(b))) for a, b in p]
        xmax = max(a for a, _ in q)
        xmin = min(a for a, _ in q)
        ymax = max(b for _, b in q)
        ymin = min(b for _, b in q)
        for slot, (cx, cy) in ((1, (xmax, ymax)), (3, (xmin, ymax)), (5, (xmin, ymin)), (7, (xmax, ymin))):
            dist = [abs(cx - a) + abs(cy - b) for a, b in q]
            best = min(range(len(q)), key=lambda i: (dist[i], i))
            assert e[slot] == best, (trial, slot)
        assert p[e[0], 0] == xmax and p[e[4], 0] == xmin
        assert p[e[2], 1] == ymax and p[e[6], 1] == ymin


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_rejected(bad):
    p = pointgen.make_points("normal", 100, seed=1)
    p[37, 1] = bad
    with pytest.raises(oracle.OracleError) as ei:
        oracle.extremes(p)
    assert ei.value.code == oracle.ERR_NONFINITE


def test_overflowing_keys_are_still_ordered():
    big = np.float32(3.0e38)
    p = np.array([(big, big), (big, 0.0), (0.0, big), (-big, -big), (-big, big)], np.float32)
    assert np.array_equal(oracle.extremes(p), brute_extremes(p))
