"""ch_filter and ch_filter_noalloc with vertex indices chosen by the caller.

The filter's contract (Sec. 3.2) is the exact "strictly inside" test for
any closed sequence of eight input points, not only for the extremes that
ch_extremes returns.  Its binary32 edge test has a static error bound
derived from the bounding box of the vertices, which holds only for points
inside that box; for caller-chosen vertices the kernels keep every point
outside the box first (such a point is never strictly inside).  These
tests hand the filter the extremes rotated by one to four slots, eight
random points, eight points near the centre, a counter-clockwise ring of
eight points at 0.3 of the data's extent, the extremes of the right half
of the data and a sequence with R and L swapped, on normal and circle inputs and on inputs with points placed on,
one ulp around, and far along the extended lines of the polygon's edges
(where a bound derived from the wrong box fails first), and compare the
survivor lists with the oracle's element by element, for both compaction
schedules and for the entry point without a workspace.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu


def _cases(p, rng):
    e = oracle.extremes(p)
    centre = np.median(p.astype(np.float64), 0)
    near_c = np.argsort(np.abs(p.astype(np.float64) - centre).sum(1))[:8].astype(np.uint32)
    swapped = e.copy()
    swapped[[0, 4]] = swapped[[4, 0]]
    out = {f"rot{k}": np.roll(e, k) for k in (1, 2, 3, 4)}
    out["random"] = rng.choice(len(p), 8, replace=False).astype(np.uint32)
    out["interior"] = near_c
    out["swap_RL"] = swapped
    # counter-clockwise polygons well inside the data: most points lie
    # outside the vertices' box, and many are discarded
    q = p.astype(np.float64) - centre
    r = 0.3 * np.abs(q).max()
    ring = [np.argmin(np.abs(q - r * np.array([np.cos(a), np.sin(a)])).sum(1)) for a in np.arange(8) * np.pi / 4]
    out["ring_ccw"] = np.array(ring, np.uint32)
    inner = np.nonzero(q[:, 0] > 0.0)[0]   # extremes of the right half
    out["half_extremes"] = inner[oracle.extremes(p[inner])].astype(np.uint32)
    return out


def _edge_points(v, m, rng, t_lo, t_hi):
    """Points a + t (b - a) on every edge line of the closed vertex sequence
    v (rounded to binary32), each with its eight one-ulp neighbours."""
    out = []
    for k in range(len(v)):
        a, b = v[k].astype(np.float64), v[(k + 1) % len(v)].astype(np.float64)
        for t in rng.uniform(t_lo, t_hi, m):
            q = (a + t * (b - a)).astype(np.float32)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    r = q.copy()
                    if dx:
                        r[0] = np.nextafter(r[0], np.float32(dx * np.inf))
                    if dy:
                        r[1] = np.nextafter(r[1], np.float32(dy * np.inf))
                    out.append(r)
    return np.array(out, np.float32).reshape(-1, 2)


def _edge_counts(n):
    m = 20 if n < 100_000 else 400
    return m, max(2, m // 4)


def _with_edge_points(base, ext, n, rng):
    """base (n minus the extra points), then points on and around the edges
    of the polygon base[ext] and far along their lines: n points in all."""
    v = base[ext]
    m_near, m_far = _edge_counts(n)
    extra = np.concatenate([_edge_points(v, m_near, rng, 0.0, 1.0), _edge_points(v, m_far, rng, -40.0, 40.0)])
    assert len(base) + len(extra) == n
    return np.ascontiguousarray(np.concatenate([base, extra]))


def _gpu_filter(d, ext, ws, how):
    n = d.shape[0]
    ext_d = torch.from_numpy(ext.view(np.int32)).cuda()
    if how == "noalloc":
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        sp = torch.full((n, 2), np.nan, dtype=torch.float32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        ch.ch_filter_noalloc(d, ext_d, idx, sp, cnt)
    else:
        ch.ch_filter_variant(0 if how == "two_pass" else 1)
        try:
            idx, sp, cnt = ch.filter_points(d, ext_d, ws)
        finally:
            ch.ch_filter_variant(0)
        torch.cuda.synchronize()
        assert ch.ch_last_error(ws.buf) == ch.CH_OK
    torch.cuda.synchronize()
    s = int(cnt.item()) & 0xFFFFFFFF
    assert s <= n, hex(s)
    return idx[:s].cpu().numpy().view(np.uint32), sp[:s].cpu().numpy()


@pytest.mark.parametrize("n", [4097, 1_000_000])
@pytest.mark.parametrize("dist", ["normal", "circle", "near_edge"])
def test_caller_vertices_match_oracle(dist, n):
    rng = np.random.default_rng(n + len(dist))
    base = pointgen.make_points("normal" if dist == "near_edge" else dist, n, seed=60 + n % 7)
    if dist == "near_edge":   # room for the points placed around each polygon's edges
        m_near, m_far = _edge_counts(n)
        base = base[: n - 8 * 9 * (m_near + m_far)]
    ws = ch.Workspace(n)
    for name, ext in _cases(base, rng).items():
        p = _with_edge_points(base, ext, n, rng) if dist == "near_edge" else base
        d = torch.from_numpy(p).cuda()
        want = oracle.filter_points(p, ext)
        for how in ("two_pass", "single_pass", "noalloc"):
            if how == "noalloc" and n > (1 << 26):
                continue
            got, gpts = _gpu_filter(d, ext, ws, how)
            assert np.array_equal(got, want), (name, how, len(got), len(want))
            assert np.array_equal(gpts.view(np.uint32), p[want].view(np.uint32)), (name, how)
