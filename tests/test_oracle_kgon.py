"""Pins of the oracle's K-direction filter polygon (the filter of the
learned proposal): with the octagon's eight integer directions it is the
octagon filter of Sec. 3.1-3.2; for other directions its vertices are the
binary32 arg-maxima recomputed by numpy, a point is discarded exactly when
rational arithmetic puts it strictly left of every edge of non-zero length,
and the hull of the survivors is the hull of all points."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import pointgen


def sets():
    out = [pointgen.make_points(d, 2000, seed=50 + i) for i, d in enumerate(pointgen.DISTRIBUTIONS)]
    rng = np.random.default_rng(4)
    g = np.array([(x, y) for x in range(-6, 7) for y in range(-6, 7)], np.float32)
    out.append(g[rng.permutation(len(g))])                                # ties everywhere
    out.append(np.full((50, 2), 1.5, np.float32))                          # one point
    t = rng.uniform(-1, 1, 200).astype(np.float32)
    out.append(np.stack([t, np.float32(2) * t], 1))                        # collinear
    out.append(pointgen.lattice_circle(25))
    return out


@pytest.mark.parametrize("k", range(7))
def test_eight_integer_directions_are_the_octagon(k):
    p = sets()[k]
    d = pointgen.kgon_directions(8)
    assert d.tolist() == [[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1]]
    assert np.array_equal(oracle.kgon_extremes(p, d), oracle.extremes(p))
    assert np.array_equal(oracle.kgon_filter(p, d), oracle.filter_points(p))


def numpy_extremes(p, d):
    x, y = p[:, 0], p[:, 1]
    out = []
    for c, s in d:
        key = (np.float32(c) * x) + (np.float32(s) * y)      # each operation rounded to binary32
        assert key.dtype == np.float32
        out.append(int(np.argmax(key)))                      # first maximum = lowest index
    return np.array(out, np.uint32)


def strictly_inside(v, q):
    """Rational check: q strictly left of every edge of non-zero length."""
    edges = 0
    qx, qy = Fraction(float(q[0])), Fraction(float(q[1]))
    for k in range(len(v)):
        a, b = v[k], v[(k + 1) % len(v)]
        if a[0] == b[0] and a[1] == b[1]:
            continue
        edges += 1
        ax, ay, bx, by = (Fraction(float(t)) for t in (a[0], a[1], b[0], b[1]))
        if (bx - ax) * (qy - ay) - (by - ay) * (qx - ax) <= 0:
            return False
    return edges > 0


@pytest.mark.parametrize("K", [3, 5, 16, 32, 64])
@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_vertices_and_discards_against_rationals(K, dist):
    p = pointgen.make_points(dist, 400, seed=K)
    d = pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=K + 1))
    e = oracle.kgon_extremes(p, d)
    assert np.array_equal(e, numpy_extremes(p, d))
    s = set(oracle.kgon_filter(p, d).tolist())
    v = p[e]
    for i in range(len(p)):
        assert (i not in s) == strictly_inside(v, p[i]), i
    assert set(e.tolist()) <= s                               # vertices are kept


@pytest.mark.parametrize("K", [8, 16, 64])
def test_hull_of_survivors_is_the_hull(K):
    for dist in pointgen.DISTRIBUTIONS:
        p = pointgen.make_points(dist, 20_000, seed=K)
        d = pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=3))
        assert np.array_equal(oracle.hull(p, oracle.kgon_filter(p, d)), oracle.hull(p))


def test_more_directions_discard_more_on_a_disc():
    # points of a disc: the 64-gon hugs the boundary more closely than the octagon
    rng = np.random.default_rng(9)
    r, th = np.sqrt(rng.uniform(0, 1, 50_000)), rng.uniform(0, 2 * np.pi, 50_000)
    p = np.stack([r * np.cos(th), r * np.sin(th)], 1).astype(np.float32)
    n8 = len(oracle.kgon_filter(p, pointgen.kgon_directions(8)))
    n64 = len(oracle.kgon_filter(p, pointgen.kgon_directions(64)))
    assert n64 < n8 / 4


def test_bad_arguments():
    p = pointgen.make_points("normal", 10, seed=1)
    with pytest.raises(oracle.OracleError):
        oracle.kgon_extremes(p, np.zeros((2, 2), np.float32))     # K < 3
    q = p.copy()
    q[3, 0] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.kgon_extremes(q, pointgen.kgon_directions(8))


def test_hand_worked_polygons():
    """tests/golden/kgon_hand_worked.json: vertices and survivors worked out
    by hand (ties, zero-length edges, points on edges and on a chord that is
    no edge)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kgon_hand_worked.json")))
    p = np.array(g["points"], np.float32)
    for case in g["cases"]:
        d = np.array(case["dirs"], np.float32)
        assert oracle.kgon_extremes(p, d).tolist() == case["vertices"], case["name"]
        assert oracle.kgon_filter(p, d).tolist() == case["survivors"], case["name"]
