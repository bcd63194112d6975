"""CPU oracle for the octagon filter and the monotone-chain hull.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module and this module never imports the product package;
the two share no code.

The arithmetic lives in ``oracle.c`` (plain sequential C, exact orientation
by a fixed-point long accumulator); this file only marshals numpy arrays.
Functions follow Algorithm 1 of Carrasco et al. (arXiv 2303.10581):

* :func:`extremes`  -- ``findingPolygon`` (Sec. 3.1)
* :func:`filter_points` -- ``buildingFilter`` + ``compactingFilteredPoints``
  (Sec. 3.2, Sec. 4.1)
* :func:`hull`      -- ``convexHull_algorithm`` (Sec. 3.3), Andrew's
  monotone chain
* :func:`convex_hull` -- the whole path
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK = 0
ERR_ARG = 1
ERR_NONFINITE = 2


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, strict IEEE binary32)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        f32 = ctypes.c_float
        p = ctypes.c_void_p
        lib.oracle_orient.argtypes = [f32] * 6
        lib.oracle_orient.restype = ctypes.c_int
        lib.oracle_set_force_exact.argtypes = [ctypes.c_int]
        lib.oracle_set_force_exact.restype = None
        lib.oracle_exact_calls.argtypes = []
        lib.oracle_exact_calls.restype = ctypes.c_uint64
        lib.oracle_extremes.argtypes = [p, ctypes.c_int64, p]
        lib.oracle_extremes.restype = ctypes.c_int
        lib.oracle_filter.argtypes = [p, ctypes.c_int64, p, p]
        lib.oracle_filter.restype = ctypes.c_int64
        lib.oracle_keep_flags.argtypes = [p, ctypes.c_int64, p, p, ctypes.c_int64, p]
        lib.oracle_keep_flags.restype = ctypes.c_int
        lib.oracle_hull.argtypes = [p, p, ctypes.c_int64, p]
        lib.oracle_kgon_extremes.argtypes = [p, ctypes.c_int64, ctypes.c_int, p, p]
        lib.oracle_kgon_extremes.restype = ctypes.c_int
        lib.oracle_kgon_filter.argtypes = [p, ctypes.c_int64, ctypes.c_int, p, p]
        lib.oracle_kgon_filter.restype = ctypes.c_int64
        lib.oracle_hull.restype = ctypes.c_int64
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def _pts(points) -> np.ndarray:
    a = np.ascontiguousarray(points, dtype=np.float32)
    if a.ndim == 1:
        a = a.reshape(-1, 2)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("points must be (n, 2) float32")
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def set_force_exact(on: bool) -> None:
    """Skip the binary64 shortcut: every orientation goes through the long accumulator."""
    _load().oracle_set_force_exact(1 if on else 0)


def exact_calls() -> int:
    """Number of orientations decided by the long accumulator so far."""
    return int(_load().oracle_exact_calls())


def orient(a, b, c) -> int:
    """Exact sign of (b - a) x (c - a) for binary32 points a, b, c."""
    f = np.float32
    return int(_load().oracle_orient(f(a[0]), f(a[1]), f(b[0]), f(b[1]), f(c[0]), f(c[1])))


def extremes(points) -> np.ndarray:
    """Indices R, TR, T, TL, L, BL, B, BR (Sec. 3.1); lowest index on ties."""
    p = _pts(points)
    if p.shape[0] == 0:
        raise ValueError("extremes of an empty set")
    out = np.zeros(8, dtype=np.uint32)
    rc = _load().oracle_extremes(_ptr(p), p.shape[0], _ptr(out))
    if rc != OK:
        raise OracleError(rc, "extremes")
    return out


def filter_points(points, ext8=None) -> np.ndarray:
    """Ascending indices of the points not strictly inside the polygon (Sec. 3.2)."""
    p = _pts(points)
    n = p.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.uint32)
    e = extremes(p) if ext8 is None else np.ascontiguousarray(ext8, dtype=np.uint32)
    out = np.empty(n, dtype=np.uint32)
    s = _load().oracle_filter(_ptr(p), n, _ptr(e), _ptr(out))
    if s < 0:
        raise OracleError(int(s), "filter")
    return out[:s].copy()


def keep_flags(points, ext8, which) -> np.ndarray:
    """Keep decision (bool) for the points listed in ``which`` only."""
    p = _pts(points)
    e = np.ascontiguousarray(ext8, dtype=np.uint32)
    w = np.ascontiguousarray(which, dtype=np.uint32)
    flags = np.zeros(w.shape[0], dtype=np.uint8)
    rc = _load().oracle_keep_flags(_ptr(p), p.shape[0], _ptr(e), _ptr(w), w.shape[0], _ptr(flags))
    if rc != OK:
        raise OracleError(rc, "keep_flags")
    return flags.astype(bool)


def hull(points, idx=None) -> np.ndarray:
    """Andrew's monotone chain over points[idx] (all points if idx is None).

    Returns original indices, counter-clockwise from the lexicographically
    smallest vertex, duplicates collapsed to the lowest index, collinear
    points excluded (Sec. 3.3)."""
    p = _pts(points)
    if idx is None:
        m = p.shape[0]
        ip = 0
        keep = None
    else:
        keep = np.ascontiguousarray(idx, dtype=np.uint32)
        m = keep.shape[0]
        ip = _ptr(keep)
    if m == 0:
        return np.zeros(0, dtype=np.uint32)
    out = np.empty(m, dtype=np.uint32)
    h = _load().oracle_hull(_ptr(p), ip, m, _ptr(out))
    if h < 0:
        raise OracleError(int(h), "hull")
    return out[:h].copy()


def kgon_extremes(points, dirs) -> np.ndarray:
    """Vertex k of the K-direction polygon: argmax of fl(fl(c_k x) + fl(s_k y))
    over the points, lowest index on ties; dirs is (K, 2) binary32."""
    p = _pts(points)
    d = np.ascontiguousarray(dirs, dtype=np.float32).reshape(-1, 2)
    out = np.zeros(d.shape[0], dtype=np.uint32)
    rc = _load().oracle_kgon_extremes(_ptr(p), p.shape[0], d.shape[0], _ptr(d), _ptr(out))
    if rc != OK:
        raise OracleError(rc, "kgon_extremes")
    return out


def kgon_filter(points, dirs, ext=None) -> np.ndarray:
    """Ascending indices of the points not strictly inside the K-vertex
    polygon of the directions dirs (or of the vertices ext)."""
    p = _pts(points)
    n = p.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.uint32)
    e = kgon_extremes(p, dirs) if ext is None else np.ascontiguousarray(ext, dtype=np.uint32)
    out = np.empty(n, dtype=np.uint32)
    s = _load().oracle_kgon_filter(_ptr(p), n, e.shape[0], _ptr(e), _ptr(out))
    if s < 0:
        raise OracleError(int(s), "kgon_filter")
    return out[:s].copy()


def convex_hull(points):
    """The whole path of Algorithm 1: (ext8, survivors, hull indices)."""
    p = _pts(points)
    if p.shape[0] == 0:
        return None, np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    e = extremes(p)
    s = filter_points(p, e)
    return e, s, hull(p, s)
