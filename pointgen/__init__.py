"""Seeded synthetic point sets shared by the tests, the smoke check and the bench.

This module holds no part of the filter or hull arithmetic: it only draws
random inputs.  Both the CUDA path and the CPU oracle consume what it makes.

Distributions (the study cases of Sec. 5 of Carrasco et al., with the
concrete parameters of the benchmark workloads):

* ``normal``    -- x, y i.i.d. Normal(0, 1) (the favourable case, Sec. 5 item 1)
* ``circle``    -- angle Uniform[0, 2 pi), point (cos, sin) on the unit circle
                   (the worst case, Sec. 5 item 2: nothing can be filtered)
* ``displaced`` -- same angle, radius 1 - |Normal(0, 0.01)| (the intermediate
                   case, Sec. 5 item 3; 0.01 is a standard deviation)

All draws are binary64 and rounded once to binary32; points are packed
(x, y) pairs, x at the lower address.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

DISTRIBUTIONS = ("normal", "circle", "displaced")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _pack(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    out = np.empty((x.shape[0], 2), dtype=np.float32)
    out[:, 0] = x
    out[:, 1] = y
    return out


def make_points(dist: str, n: int, seed: int, chunk: int = 1 << 24) -> np.ndarray:
    """(n, 2) float32 points of one distribution, reproducible from ``seed``.

    Large n is produced in chunks from one stream so memory stays bounded."""
    if dist not in DISTRIBUTIONS:
        raise ValueError(f"unknown distribution {dist!r}")
    rng = _rng(seed)
    out = np.empty((n, 2), dtype=np.float32)
    for lo in range(0, n, chunk):
        m = min(chunk, n - lo)
        if dist == "normal":
            out[lo:lo + m, 0] = rng.standard_normal(m)
            out[lo:lo + m, 1] = rng.standard_normal(m)
        else:
            theta = rng.uniform(0.0, 2.0 * math.pi, m)
            if dist == "circle":
                r = 1.0
            else:
                r = 1.0 - np.abs(rng.normal(0.0, 0.01, m))
            out[lo:lo + m, 0] = r * np.cos(theta)
            out[lo:lo + m, 1] = r * np.sin(theta)
    return out


def _fill_blocks(fn, nblocks: int, workers: int | None):
    """fn(b) for b < nblocks, on `workers` threads (numpy's generators and
    ufuncs release the GIL); each block draws from its own generator, so
    the result does not depend on the thread count."""
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1:
        for b in range(nblocks):
            fn(b)
        return
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(fn, range(nblocks)))


def make_points_blocked(dist: str, n: int, seed: int, block: int = 1 << 24, workers: int | None = None) -> np.ndarray:
    """(n, 2) float32 points of one distribution, like make_points, but block
    k of `block` points draws from its own stream (SeedSequence(seed)
    spawned once per block), so large sets are generated on several threads
    and the result still depends only on (dist, n, seed, block)."""
    if dist not in DISTRIBUTIONS:
        raise ValueError(f"unknown distribution {dist!r}")
    nblocks = (n + block - 1) // block
    seqs = np.random.SeedSequence(seed).spawn(max(nblocks, 1))
    out = np.empty((n, 2), dtype=np.float32)

    def fill(b):
        lo = b * block
        m = min(block, n - lo)
        rng = np.random.Generator(np.random.PCG64(seqs[b]))
        if dist == "normal":
            out[lo:lo + m, 0] = rng.standard_normal(m)
            out[lo:lo + m, 1] = rng.standard_normal(m)
        else:
            theta = rng.uniform(0.0, 2.0 * math.pi, m)
            r = 1.0 if dist == "circle" else 1.0 - np.abs(rng.normal(0.0, 0.01, m))
            out[lo:lo + m, 0] = r * np.cos(theta)
            out[lo:lo + m, 1] = r * np.sin(theta)

    _fill_blocks(fill, nblocks, workers)
    return out


def make_batch(num_sets: int, seed: int, min_n: int = 100, max_n: int = 1_000_000, workers: int | None = None):
    """Independent sets of uneven sizes, concatenated in CSR form.

    Sizes are log-uniform in [min_n, max_n]; each set draws its distribution
    uniformly from the three above, is scaled by Uniform[0.1, 10] and rotated
    by Uniform[0, 2 pi) (in binary64, then rounded to binary32).  Every set
    has its own generator (seeded from the batch's), so the sets are filled
    on `workers` threads with the same result.
    Returns (points (N, 2) float32, offsets (num_sets + 1,) int64, dists list).
    """
    rng = _rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(min_n), math.log(max_n), num_sets))).astype(np.int64)
    kinds = rng.integers(0, 3, num_sets)
    scales = rng.uniform(0.1, 10.0, num_sets)
    angles = rng.uniform(0.0, 2.0 * math.pi, num_sets)
    sub_seeds = rng.integers(0, 2**62, num_sets)
    offsets = np.zeros(num_sets + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    pts = np.empty((int(offsets[-1]), 2), dtype=np.float32)
    dists = [DISTRIBUTIONS[int(k)] for k in kinds]

    def fill(b):
        dist = dists[b]
        r2 = _rng(int(sub_seeds[b]))
        m = int(sizes[b])
        if dist == "normal":
            x = r2.standard_normal(m)
            y = r2.standard_normal(m)
        else:
            th = r2.uniform(0.0, 2.0 * math.pi, m)
            r = 1.0 if dist == "circle" else 1.0 - np.abs(r2.normal(0.0, 0.01, m))
            x = r * np.cos(th)
            y = r * np.sin(th)
        c, s = math.cos(angles[b]), math.sin(angles[b])
        sc = scales[b]
        pts[offsets[b]:offsets[b + 1], 0] = sc * (c * x - s * y)
        pts[offsets[b]:offsets[b + 1], 1] = sc * (s * x + c * y)

    _fill_blocks(fill, num_sets, workers)
    return pts, offsets, dists


def lattice_circle(radius: int) -> np.ndarray:
    """All integer points (x, y) with x^2 + y^2 = radius^2, in a fixed
    (not hull) order: ascending x, then ascending y.  Exact in binary32 for
    radius < 2^24."""
    pts = []
    r2 = radius * radius
    for x in range(-radius, radius + 1):
        y2 = r2 - x * x
        y = math.isqrt(y2)
        if y * y == y2:
            if y == 0:
                pts.append((x, 0))
            else:
                pts.append((x, -y))
                pts.append((x, y))
    return np.array(pts, dtype=np.float32).reshape(-1, 2)


# the eight integer directions of the octagon, counter-clockwise from +x
_OCTAGON_DIRS = ((1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1))


def kgon_directions(K: int, offsets=None) -> np.ndarray:
    """(K, 2) binary32 directions (c_k, s_k) at the angles 2 pi k / K + off_k,
    counter-clockwise: an input of the K-direction filter polygon (the
    parameters a learned proposal would choose).  cos and sin are taken in
    binary64 and rounded once; an angle that is a multiple of pi/4 with zero
    offset gets the octagon's integer direction instead, so K = 8 without
    offsets gives the octagon's keys exactly."""
    off = np.zeros(K) if offsets is None else np.asarray(offsets, dtype=np.float64)
    out = np.empty((K, 2), dtype=np.float32)
    for k in range(K):
        if off[k] == 0.0 and (8 * k) % K == 0:
            out[k] = _OCTAGON_DIRS[8 * k // K]
        else:
            th = 2.0 * math.pi * k / K + float(off[k])
            out[k] = (math.cos(th), math.sin(th))
    return out


def kgon_offsets(K: int, seed: int, spread: float = 0.45) -> np.ndarray:
    """Random angular offsets in (-spread, spread) * pi / K: the directions
    stay in counter-clockwise order."""
    return (_rng(seed).uniform(-spread, spread, K) * math.pi / K).astype(np.float64)


FAMILIES = ("gaussians", "ellipse", "displaced")


def make_family(kind: str, n: int, seed: int) -> np.ndarray:
    """(n, 2) float32 points of one of the learned proposal's training
    families, randomly scaled and rotated:
    ``gaussians`` a mixture of 1-4 anisotropic Gaussians; ``ellipse`` points
    near an ellipse with axis ratio Uniform[1, 20] (radius factor
    1 - |Normal(0, 0.01)|); ``displaced`` the displaced circle."""
    rng = _rng(seed)
    if kind == "gaussians":
        comps = int(rng.integers(1, 5))
        which = rng.integers(0, comps, n)
        means = rng.uniform(-3.0, 3.0, (comps, 2))
        sig = rng.uniform(0.1, 1.0, (comps, 2))
        rot = rng.uniform(0.0, 2.0 * math.pi, comps)
        z = rng.standard_normal((n, 2)) * sig[which]
        c, s = np.cos(rot[which]), np.sin(rot[which])
        x = means[which, 0] + c * z[:, 0] - s * z[:, 1]
        y = means[which, 1] + s * z[:, 0] + c * z[:, 1]
    else:
        th = rng.uniform(0.0, 2.0 * math.pi, n)
        r = 1.0 - np.abs(rng.standard_normal(n)) * 0.01
        ratio = rng.uniform(1.0, 20.0) if kind == "ellipse" else 1.0
        u, v = r * np.cos(th), r * np.sin(th) / ratio
        a = rng.uniform(0.0, 2.0 * math.pi)
        x, y = math.cos(a) * u - math.sin(a) * v, math.sin(a) * u + math.cos(a) * v
    scale = rng.uniform(0.1, 10.0)
    return _pack(x * scale, y * scale)
