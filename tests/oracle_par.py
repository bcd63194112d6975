"""Running the oracle over very large inputs in reasonable time.

Test infrastructure: the oracle's functions are called unchanged, only on
disjoint pieces of the work, from threads (ctypes releases the GIL for the
duration of a foreign call, so the pieces run on separate cores).

* The filter's keep decision is per point (Sec. 3.2): the survivors of the
  whole set are the union of the survivors of disjoint index ranges, each
  decided against the same eight vertices (``oracle.keep_flags``).
* The K-direction filter is per point too: each range is filtered as its
  own array with the K vertices' coordinates placed in front of it (the
  decision depends only on those coordinates and on the point).
* The hull of a set is the hull of the union of the hulls of any split of
  it (Sec. 3.3: a hull vertex of the whole set is a strictly convex extreme
  point, hence a vertex of the hull of every part holding it, and its
  lowest index lies in one of the parts), so the parts' hulls are computed
  in threads and the oracle's hull runs once more over their union.
* Independent point sets (a batch) are independent oracle calls.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def filter_points(p: np.ndarray, ext8: np.ndarray, chunk: int = 1 << 24) -> np.ndarray:
    """oracle.filter_points(p, ext8), computed range by range in threads."""
    n = len(p)
    ext8 = np.ascontiguousarray(ext8, np.uint32)

    def piece(lo):
        hi = min(n, lo + chunk)
        which = np.arange(lo, hi, dtype=np.uint32)
        return which[oracle.keep_flags(p, ext8, which)]

    with ThreadPoolExecutor(threads()) as ex:
        parts = list(ex.map(piece, range(0, n, chunk)))
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def kgon_filter(p: np.ndarray, dirs: np.ndarray, ext: np.ndarray, chunk: int = 1 << 23) -> np.ndarray:
    """oracle.kgon_filter(p, dirs, ext), computed range by range in threads."""
    n = len(p)
    ext = np.ascontiguousarray(ext, np.uint32)
    K = len(ext)
    verts = p[ext]

    def piece(lo):
        hi = min(n, lo + chunk)
        q = np.concatenate([verts, p[lo:hi]])
        s = oracle.kgon_filter(q, dirs, np.arange(K, dtype=np.uint32)).astype(np.int64)
        return (s[s >= K] - K + lo).astype(np.uint32)

    with ThreadPoolExecutor(threads()) as ex:
        parts = list(ex.map(piece, range(0, n, chunk)))
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def hull(p: np.ndarray, idx: np.ndarray, parts: int | None = None) -> np.ndarray:
    """oracle.hull(p, idx), from the hulls of `parts` pieces of idx."""
    idx = np.ascontiguousarray(idx, np.uint32)
    parts = parts or threads()
    if len(idx) < 4 * parts:
        return oracle.hull(p, idx)
    pieces = np.array_split(idx, parts)
    with ThreadPoolExecutor(threads()) as ex:
        hulls = list(ex.map(lambda q: oracle.hull(p, q), pieces))
    return oracle.hull(p, np.sort(np.concatenate(hulls)))


def map_sets(fn, items):
    """[fn(x) for x in items], the calls spread over threads."""
    with ThreadPoolExecutor(threads()) as ex:
        return list(ex.map(fn, items))
