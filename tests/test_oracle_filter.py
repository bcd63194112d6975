"""Pins for the oracle's filter (Sec. 3.2 buildingFilter + compaction).

Every discarded point must lie strictly inside the polygon and every kept
point must not (both re-checked on exact rationals); the eight vertices are
always kept; the survivor list is ascending; discarding never changes the
hull (brute force on small sets); points on a circle are never discarded.
"""
import numpy as np
import pytest

import oracle
import pointgen
from exact_ref import brute_hull, strictly_inside_q


def _check_filter_exact(p):
    e = oracle.extremes(p)
    s = oracle.filter_points(p, e)
    poly = [p[i] for i in e]
    kept = np.zeros(len(p), bool)
    kept[s] = True
    assert np.all(np.diff(s.astype(np.int64)) > 0)
    for i in range(len(p)):
        assert kept[i] == (not strictly_inside_q(poly, p[i])), i
    assert np.all(kept[e])
    return e, s


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_filter_matches_exact_definition(dist):
    p = pointgen.make_points(dist, 1500, seed=21)
    _check_filter_exact(p)


def test_filter_on_grid_with_boundary_points():
    # integer grid: many points exactly on polygon edges, which must be kept
    g = np.array([(x, y) for x in range(-6, 7) for y in range(-6, 7) if abs(x) + abs(y) <= 9], np.float32)
    rng = np.random.default_rng(5)
    p = g[rng.permutation(len(g))]
    _, s = _check_filter_exact(p)
    assert 0 < len(s) < len(p)


def test_filter_degenerate_sets_keep_everything():
    for p in (
        np.full((10, 2), 1.5, np.float32),
        np.array([(k, 2 * k) for k in range(20)], np.float32),
        np.array([(0, 0), (1, 0)], np.float32),
        np.array([(0, 0)], np.float32),
    ):
        assert len(oracle.filter_points(p)) == len(p)


def test_lattice_circle_keeps_everything():
    p = pointgen.lattice_circle(1105)
    assert len(oracle.filter_points(p)) == len(p)


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_hull_of_survivors_is_hull_of_all(dist):
    for seed in range(3):
        p = pointgen.make_points(dist, 60, seed=100 + seed)
        e, s, h = oracle.convex_hull(p)
        assert list(h) == brute_hull(p)
        assert list(oracle.hull(p)) == list(h)


def test_normal_filters_most_points():
    p = pointgen.make_points("normal", 200_000, seed=1)
    s = oracle.filter_points(p)
    assert len(s) < 2000


def test_circle_filters_nothing():
    p = pointgen.make_points("circle", 200_000, seed=1)
    assert len(oracle.filter_points(p)) == len(p)


def test_keep_flags_agree_with_filter():
    p = pointgen.make_points("displaced", 5000, seed=2)
    e = oracle.extremes(p)
    s = oracle.filter_points(p, e)
    which = np.arange(len(p), dtype=np.uint32)
    f = oracle.keep_flags(p, e, which)
    assert np.array_equal(np.nonzero(f)[0].astype(np.uint32), s)


def _vertex_sequences(p, rng):
    """Vertex index sequences a caller may hand the filter: the extremes
    rotated, eight random points, eight points near the centre, R and L
    swapped, and a sequence with repeats."""
    e = oracle.extremes(p)
    c = np.argsort(np.abs(p.astype(np.float64) - np.median(p, 0)).sum(1))[:8]
    swapped = e.copy()
    swapped[[0, 4]] = swapped[[4, 0]]
    return {
        "rot1": np.roll(e, 1), "rot3": np.roll(e, 3), "rot4": np.roll(e, 4),
        "random": rng.choice(len(p), 8, replace=False).astype(np.uint32),
        "interior": c.astype(np.uint32),
        "swap_RL": swapped,
        "repeats": np.array([e[0], e[0], e[2], e[2], e[2], e[4], e[6], e[6]], np.uint32),
    }


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_filter_any_vertex_sequence_matches_exact_definition(dist):
    """The filter's definition holds for any eight vertices, not only for
    the extremes: discarded <=> strictly left of every edge of non-zero
    length (rationals), whatever the order or position of the vertices."""
    rng = np.random.default_rng(23)
    p = pointgen.make_points(dist, 700, seed=24)
    for name, ext in _vertex_sequences(p, rng).items():
        s = oracle.filter_points(p, ext)
        poly = [p[i] for i in ext]
        kept = np.zeros(len(p), bool)
        kept[s] = True
        for i in range(len(p)):
            assert kept[i] == (not strictly_inside_q(poly, p[i])), (name, i)
