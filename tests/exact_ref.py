"""Exact rational reference helpers for the tests (Python ``fractions``).

Independent of both the oracle's C code and the CUDA path: orientation is
the textbook 2x2 determinant evaluated on exact rationals, and the hull is
the brute-force edge test (an ordered pair (i, j) is a counter-clockwise
hull edge when no point lies strictly to its right and every point on its
line lies on the closed segment).  Only practical for small inputs.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def F(v) -> Fraction:
    return Fraction(float(np.float32(v)))


def orient_q(a, b, c) -> int:
    ax, ay, bx, by, cx, cy = (F(v) for v in (a[0], a[1], b[0], b[1], c[0], c[1]))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def strictly_inside_q(poly, p) -> bool:
    """p strictly left of every non-degenerate edge of the closed sequence poly."""
    m = len(poly)
    edges = 0
    for k in range(m):
        a, b = poly[k], poly[(k + 1) % m]
        if F(a[0]) == F(b[0]) and F(a[1]) == F(b[1]):
            continue
        edges += 1
        if orient_q(a, b, p) <= 0:
            return False
    return edges > 0


def _dedupe_lowest(pts, idx):
    seen = {}
    for i in idx:
        key = (F(pts[i][0]), F(pts[i][1]))
        if key not in seen or i < seen[key]:
            seen[key] = i
    return sorted(seen.values())


def brute_hull(pts, idx=None):
    """Counter-clockwise hull vertex indices from the lexicographically
    smallest vertex; equal points collapse to the lowest index; collinear
    points are not vertices."""
    pts = np.asarray(pts, dtype=np.float32)
    cand = list(range(len(pts))) if idx is None else [int(i) for i in idx]
    if not cand:
        return []
    u = _dedupe_lowest(pts, cand)
    if len(u) == 1:
        return [u[0]]
    q = {i: (F(pts[i][0]), F(pts[i][1])) for i in u}

    def on_segment(i, j, k):
        (xi, yi), (xj, yj), (xk, yk) = q[i], q[j], q[k]
        return min(xi, xj) <= xk <= max(xi, xj) and min(yi, yj) <= yk <= max(yi, yj)

    def orient(i, j, k):
        (xi, yi), (xj, yj), (xk, yk) = q[i], q[j], q[k]
        d = (xj - xi) * (yk - yi) - (yj - yi) * (xk - xi)
        return (d > 0) - (d < 0)

    nxt = {}
    for i in u:
        for j in u:
            if i == j:
                continue
            ok = True
            for k in u:
                if k == i or k == j:
                    continue
                o = orient(i, j, k)
                if o < 0 or (o == 0 and not on_segment(i, j, k)):
                    ok = False
                    break
            if ok:
                assert i not in nxt, "two outgoing hull edges"
                nxt[i] = j
    start = min(u, key=lambda i: (q[i][0], q[i][1]))
    out = [start]
    cur = nxt[start]
    while cur != start:
        out.append(cur)
        cur = nxt[cur]
        assert len(out) <= len(u)
    return out


def strictly_convex_ccw(pts, hull) -> bool:
    h = len(hull)
    if h < 3:
        return True
    for k in range(h):
        if orient_q(pts[hull[k]], pts[hull[(k + 1) % h]], pts[hull[(k + 2) % h]]) <= 0:
            return False
    return True
