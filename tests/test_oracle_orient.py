"""Pins for the oracle's exact orientation predicate.

The oracle decides the sign of (b - a) x (c - a) for binary32 inputs with a
long accumulator (plus a binary64 shortcut guarded by the recursive
summation bound).  These tests pin it to exact rational arithmetic on
random, wide-range and adversarial near-collinear triples, and check that
the shortcut and the accumulator agree.
"""
import numpy as np
import pytest

import oracle
from exact_ref import orient_q


def _wide_floats(rng, m):
    """binary32 values spread over the whole exponent range, incl. subnormals."""
    exp = rng.integers(-149, 127, m)
    mant = rng.uniform(1.0, 2.0, m)
    v = (mant * np.exp2(exp.astype(np.float64))).astype(np.float32)
    sign = np.where(rng.random(m) < 0.5, -1.0, 1.0).astype(np.float32)
    return v * sign


def _near_collinear(rng, m, scale):
    """c on the line through a and b (rounded), then nudged by a few ulps."""
    out = []
    for _ in range(m):
        a = (rng.standard_normal(2) * scale).astype(np.float32)
        b = (rng.standard_normal(2) * scale).astype(np.float32)
        t = rng.uniform(-2.0, 3.0)
        c = (a.astype(np.float64) + t * (b.astype(np.float64) - a.astype(np.float64))).astype(np.float32)
        k = int(rng.integers(-2, 3))
        axis = int(rng.integers(0, 2))
        for _ in range(abs(k)):
            c[axis] = np.nextafter(c[axis], np.float32(np.inf) if k > 0 else np.float32(-np.inf))
        out.append((a, b, c))
    return out


def test_basic_signs():
    assert oracle.orient((0, 0), (1, 0), (0, 1)) == 1
    assert oracle.orient((0, 0), (1, 0), (0, -1)) == -1
    assert oracle.orient((0, 0), (1, 0), (7, 0)) == 0
    assert oracle.orient((3, 3), (3, 3), (1, 2)) == 0


@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e30, 1e-42])
def test_near_collinear_matches_rational(scale):
    rng = np.random.default_rng(11)
    for a, b, c in _near_collinear(rng, 400, scale):
        assert oracle.orient(a, b, c) == orient_q(a, b, c), (a, b, c)


def test_wide_range_matches_rational():
    rng = np.random.default_rng(12)
    v = _wide_floats(rng, 6 * 2000).reshape(-1, 6)
    for r in v:
        a, b, c = r[0:2], r[2:4], r[4:6]
        assert oracle.orient(a, b, c) == orient_q(a, b, c)


def test_extreme_magnitudes():
    big = np.float32(3.4e38)
    tiny = np.float32(1.4e-45)
    cases = [
        ((-big, -big), (big, big), (big, -big)),
        ((-big, -big), (big, big), (np.nextafter(big, np.float32(0)), big)),
        ((0, 0), (tiny, tiny), (2 * tiny, 2 * tiny)),
        ((0, 0), (tiny, tiny), (2 * tiny, tiny)),
        ((tiny, 0), (0, tiny), (-big, big)),
        ((1.0, 1.0), (1.0 + 2**-23, 1.0 + 2**-23), (1e30, 1e30)),
        ((1.0, 1.0), (1.0 + 2**-23, 1.0 + 2**-23), (1e30, np.nextafter(np.float32(1e30), np.float32(0)))),
    ]
    for a, b, c in cases:
        a = np.array(a, np.float32)
        b = np.array(b, np.float32)
        c = np.array(c, np.float32)
        assert oracle.orient(a, b, c) == orient_q(a, b, c), (a, b, c)


def test_symmetries():
    rng = np.random.default_rng(13)
    for a, b, c in _near_collinear(rng, 300, 1.0):
        s = oracle.orient(a, b, c)
        assert oracle.orient(b, c, a) == s
        assert oracle.orient(c, a, b) == s
        assert oracle.orient(b, a, c) == -s
        assert oracle.orient(a, c, b) == -s


def test_shortcut_agrees_with_accumulator():
    rng = np.random.default_rng(14)
    triples = _near_collinear(rng, 300, 1.0)
    v = _wide_floats(rng, 6 * 300).reshape(-1, 6)
    triples += [(r[0:2], r[2:4], r[4:6]) for r in v]
    fast = [oracle.orient(a, b, c) for a, b, c in triples]
    before = oracle.exact_calls()
    oracle.set_force_exact(True)
    try:
        exact = [oracle.orient(a, b, c) for a, b, c in triples]
    finally:
        oracle.set_force_exact(False)
    assert oracle.exact_calls() - before == len(triples)
    assert fast == exact


def test_accumulator_is_reached_by_degenerate_cases():
    """Exactly collinear triples and heavy cancellation far from the origin
    must be decided by the long accumulator, and still match the rationals."""
    rng = np.random.default_rng(15)
    before = oracle.exact_calls()
    for _ in range(200):
        a = rng.integers(-1000, 1000, 2)
        d = rng.integers(-50, 50, 2)
        t = int(rng.integers(-5, 6))
        tri = (a, a + d, a + t * d)
        tri = tuple(np.asarray(v, np.float32) for v in tri)
        assert oracle.orient(*tri) == 0 == orient_q(*tri)
    base = np.float32(2.0**30)
    for _ in range(200):
        off = rng.integers(-64, 64, 6).astype(np.float32)
        a = (base + off[0], base + off[1])
        b = (base + off[2], base + off[3])
        c = (base + off[4], base + off[5])
        assert oracle.orient(a, b, c) == orient_q(a, b, c)
    assert oracle.exact_calls() - before >= 300
