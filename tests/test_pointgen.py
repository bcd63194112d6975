"""The input generators: reproducible from their seeds whatever the number
of threads that fill them, with the distributions' defining properties."""
import numpy as np

import pointgen


def test_batch_does_not_depend_on_threads():
    a, oa, da = pointgen.make_batch(200, seed=5, workers=1)
    b, ob, db = pointgen.make_batch(200, seed=5, workers=7)
    assert np.array_equal(oa, ob) and da == db
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_blocked_points_do_not_depend_on_threads():
    for dist in pointgen.DISTRIBUTIONS:
        a = pointgen.make_points_blocked(dist, 300_007, seed=3, block=1 << 14, workers=1)
        b = pointgen.make_points_blocked(dist, 300_007, seed=3, block=1 << 14, workers=5)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_blocked_points_follow_their_distribution():
    p = pointgen.make_points_blocked("normal", 1 << 20, seed=4, block=1 << 16).astype(np.float64)
    assert abs(p.mean()) < 0.01 and abs(p.std() - 1.0) < 0.01
    c = pointgen.make_points_blocked("circle", 1 << 16, seed=4).astype(np.float64)
    assert np.allclose(np.hypot(c[:, 0], c[:, 1]), 1.0, atol=1e-6)
    d = pointgen.make_points_blocked("displaced", 1 << 16, seed=4).astype(np.float64)
    r = np.hypot(d[:, 0], d[:, 1])
    assert r.max() <= 1.0 + 1e-6 and abs((1.0 - r).mean() - 0.01 * np.sqrt(2 / np.pi)) < 5e-4
