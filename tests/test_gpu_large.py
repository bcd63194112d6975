"""Oracle parity at the largest workloads: 10^9 normal points (extremes,
both compaction schedules, the hull), the whole 4096-set batch (every
set's hull) and the learned K-gon path on 10^8-point sets of its three
families (survivors of the chosen polygon and the hull), in the launch
configurations the benchmark uses.  Every output is an index list, so the
comparison is element by element.

The oracle runs unchanged; only its work is spread over threads (per-point
keep decisions over disjoint index ranges, hulls of parts then of their
union, independent sets), see oracle_par."""
import numpy as np
import pytest
import torch

import oracle
import oracle_par
import paper_2303_10581_gb300 as ch
import pointgen
from paper_2303_10581_gb300 import learned

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _u32(t, k=None):
    a = t.cpu().numpy() if k is None else t[:k].cpu().numpy()
    return a.view(np.uint32)


def test_normal_1e9_both_schedules_and_hull():
    n = 1_000_000_000
    p = pointgen.make_points_blocked("normal", n, seed=1)   # the benchmark's 10^9-point set
    d = torch.from_numpy(p).cuda()
    ws = ch.Workspace(n)
    ext = ch.extremes(d, ws)
    e = _u32(ext)
    assert np.array_equal(e, oracle.extremes(p))
    want = oracle_par.filter_points(p, e)
    assert 0 < len(want) < 1000
    for variant in (0, 1):
        ch.ch_filter_variant(variant)
        try:
            idx, sp, cnt = ch.filter_points(d, ext, ws)
            ws.check()
        finally:
            ch.ch_filter_variant(0)
        s = int(cnt.item())
        assert np.array_equal(_u32(idx, s), want), variant
        assert np.array_equal(sp[:s].cpu().numpy().view(np.uint32), p[want].view(np.uint32))
        del idx, sp
    hidx, hcnt = ch.convex_hull(d, ws)
    ws.check()
    assert np.array_equal(_u32(hidx, int(hcnt.item())), oracle.hull(p, want))
    del d, ws, hidx, ext
    _free()


def test_batch_4096_sets_every_hull():
    B = 4096
    pts, off, _ = pointgen.make_batch(B, seed=1)
    n = len(pts)
    d = torch.from_numpy(pts).cuda()
    ws = ch.Workspace(n, num_sets=B)
    hidx, hoff = ch.convex_hull_batched(d, torch.from_numpy(off).cuda(), ws)
    ws.check()
    got_off = hoff.cpu().numpy()
    got = hidx.cpu().numpy().view(np.uint32)
    want = oracle_par.map_sets(lambda b: oracle.convex_hull(pts[off[b]:off[b + 1]])[2], range(B))
    assert np.array_equal(np.diff(got_off), [len(w) for w in want])
    for b in range(B):
        assert np.array_equal(got[got_off[b]:got_off[b + 1]], want[b]), b
    del d, ws, hidx
    _free()


@pytest.mark.parametrize("kind", pointgen.FAMILIES)
def test_learned_path_1e8(kind):
    """The proposal's polygon (an untrained proposal picks some K and
    offsets; results must not depend on the choice) and two fixed ones:
    survivors against the oracle's K-direction filter, hulls against the
    oracle's hull and the octagon path's."""
    n = 100_000_000
    p = pointgen.make_family(kind, n, seed=7 + pointgen.FAMILIES.index(kind))
    e = oracle.extremes(p)
    want_hull = oracle_par.hull(p, oracle_par.filter_points(p, e))
    d = torch.from_numpy(p).cuda()
    ws = ch.Workspace(n)
    prop = learned.Proposal(seed=3)
    K, units = prop.propose(d)
    choices = [(K, units), (16, np.zeros(16)), (64, pointgen.kgon_offsets(64, seed=5) * 64 / np.pi)]
    for K, u in choices:
        dirs = learned.directions(K, u)
        vert, idx, _, cnt = ch.filter_points_kgon(d, dirs, ws)
        ws.check()
        s = int(cnt.item())
        v = _u32(vert)
        assert np.array_equal(v, oracle.kgon_extremes(p, dirs)), K
        assert np.array_equal(_u32(idx, s), oracle_par.kgon_filter(p, dirs, v)), K
        hidx, hcnt = ch.convex_hull_kgon(d, dirs, ws)
        ws.check()
        assert np.array_equal(_u32(hidx, int(hcnt.item())), want_hull), K
        del idx, hidx
    lidx, lcnt, _ = prop.hull(d, ws)
    ws.check()
    assert np.array_equal(_u32(lidx, int(lcnt.item())), want_hull)
    hidx, hcnt = ch.convex_hull(d, ws)
    ws.check()
    assert np.array_equal(_u32(hidx, int(hcnt.item())), want_hull)
    del d, ws, lidx, hidx
    _free()
