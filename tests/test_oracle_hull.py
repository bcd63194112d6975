"""Pins for the oracle's hull (Sec. 3.3, Andrew's monotone chain) and for the
whole path on hand-worked fixtures.

Brute-force O(n^3) hulls on exact rationals for tiny sets (with duplicates
and collinear points), closed forms (lattice points on a circle, square
corners, collinear sets), and the hand-worked cases in tests/golden/.
"""
import json
import os

import numpy as np
import pytest

import oracle
import pointgen
from exact_ref import brute_hull, strictly_convex_ccw

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _load("hand_worked.json")["cases"], ids=lambda c: c["name"])
def test_hand_worked_cases(case):
    p = np.array(case["points"], np.float32)
    e, s, h = oracle.convex_hull(p)
    assert list(e) == case["ext8"]
    assert list(s) == case["survivors"]
    assert list(h) == case["hull"]


@pytest.mark.parametrize("case", _load("lattice_circles.json")["cases"], ids=lambda c: str(c["radius"]))
def test_lattice_circle_closed_form(case):
    p = pointgen.lattice_circle(case["radius"])
    assert len(p) == case["count"]
    rng = np.random.default_rng(case["radius"])
    p = p[rng.permutation(len(p))]
    e, s, h = oracle.convex_hull(p)
    assert len(s) == case["count"]
    assert len(h) == case["count"]
    assert strictly_convex_ccw(p, h)
    first = p[h[0]]
    assert first[0] == -case["radius"] and first[1] == 0


def test_square_corners_with_interior_points():
    rng = np.random.default_rng(8)
    inner = rng.uniform(-0.99, 0.99, size=(5000, 2)).astype(np.float32)
    corners = np.array([(1, 1), (-1, 1), (-1, -1), (1, -1)], np.float32)
    p = np.concatenate([inner[:2500], corners, inner[2500:]])
    h = oracle.convex_hull(p)[2]
    got = [tuple(p[i]) for i in h]
    assert got == [(-1, -1), (1, -1), (1, 1), (-1, 1)]


def test_collinear_hull_is_two_endpoints():
    t = np.linspace(-3, 5, 41).astype(np.float32)
    p = np.stack([t, np.float32(0.5) * t], axis=1)
    rng = np.random.default_rng(2)
    p = p[rng.permutation(len(p))]
    h = oracle.hull(p)
    assert [tuple(p[i]) for i in h] == [tuple(p[np.argmin(p[:, 0])]), tuple(p[np.argmax(p[:, 0])])]


def test_single_and_double_points():
    assert list(oracle.hull(np.array([(2, 3)], np.float32))) == [0]
    assert list(oracle.hull(np.array([(2, 3), (2, 3)], np.float32))) == [0]
    assert list(oracle.hull(np.array([(5, 3), (2, 3)], np.float32))) == [1, 0]
    assert list(oracle.hull(np.zeros((0, 2), np.float32))) == []


@pytest.mark.parametrize("seed", range(25))
def test_matches_brute_force_on_degenerate_small_sets(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 28))
    kind = seed % 3
    if kind == 0:
        p = rng.integers(-3, 4, size=(n, 2)).astype(np.float32)   # grid: duplicates, collinear
    elif kind == 1:
        p = rng.standard_normal((n, 2)).astype(np.float32)
    else:
        t = rng.integers(-4, 5, n).astype(np.float32)
        p = np.stack([t, 2 * t + rng.integers(0, 2, n)], axis=1).astype(np.float32)
    assert list(oracle.hull(p)) == brute_hull(p)
    e, s, h = oracle.convex_hull(p)
    assert list(h) == brute_hull(p)


def test_signed_zero_is_one_point():
    p = np.array([(0.0, 0.0), (-0.0, 0.0), (1, 0), (0, 1), (0.0, -0.0)], np.float32)
    assert list(oracle.hull(p)) == [0, 2, 3]


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_hull_invariants_medium(dist):
    p = pointgen.make_points(dist, 20000, seed=4)
    e, s, h = oracle.convex_hull(p)
    assert len(h) <= len(s) <= len(p)
    assert strictly_convex_ccw(p, h)
    assert set(h.tolist()) <= set(s.tolist())
    # hull of everything equals hull of the survivors
    assert np.array_equal(oracle.hull(p), h)
