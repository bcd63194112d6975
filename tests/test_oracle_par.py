"""The threaded oracle helpers give exactly the oracle's results: the same
survivor lists (octagon and K-direction polygons) and the same hulls,
including inputs with duplicates and collinear points, where the split
into parts must not change which index represents a point."""
import numpy as np
import pytest

import oracle
import oracle_par
import pointgen


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_filter_and_hull_match_the_oracle(dist):
    p = pointgen.make_points(dist, 300_001, seed=71)
    e = oracle.extremes(p)
    s = oracle.filter_points(p, e)
    assert np.array_equal(oracle_par.filter_points(p, e, chunk=4096 + 3), s)
    assert np.array_equal(oracle_par.hull(p, s, parts=7), oracle.hull(p, s))


def test_hull_with_duplicates_and_collinear_points():
    rng = np.random.default_rng(72)
    base = pointgen.make_points("circle", 2000, seed=73)
    square = np.array([(x, y) for x in range(-3, 4) for y in range(-3, 4)], np.float32)
    p = np.concatenate([base[rng.integers(0, 2000, 30_000)], square * np.float32(0.5)])
    p = p[rng.permutation(len(p))]
    idx = np.arange(len(p), dtype=np.uint32)
    assert np.array_equal(oracle_par.hull(p, idx, parts=9), oracle.hull(p, idx))


@pytest.mark.parametrize("K", [8, 16, 64])
def test_kgon_filter_matches_the_oracle(K):
    p = pointgen.make_family("ellipse", 200_003, seed=74)
    dirs = pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=75))
    v = oracle.kgon_extremes(p, dirs)
    assert np.array_equal(oracle_par.kgon_filter(p, dirs, v, chunk=5000), oracle.kgon_filter(p, dirs, v))
