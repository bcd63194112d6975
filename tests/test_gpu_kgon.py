"""GPU parity of the K-direction filter polygon (ch_filter_kgon,
ch_hull_kgon) against the oracle: vertex indices, survivor lists and
coordinates, and hulls bit for bit, for K = 8, 16, 32, 64 with random
angular offsets, over sizes with ragged tiles, degenerate sets, an
8-byte-aligned view and a non-finite coordinate; with the octagon's eight
integer directions it must equal ch_filter."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu


def dev(p):
    return torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()


def run_filter(d, dirs, ws=None):
    ws = ws or ch.Workspace(max(d.shape[0], 1))
    ext, idx, sp, cnt = ch.filter_points_kgon(d, dirs, ws)
    torch.cuda.synchronize()
    status = ch.ch_last_error(ws.buf)
    s = int(cnt.item())
    return (status, ext.cpu().numpy().view(np.uint32), idx[:s].cpu().numpy().view(np.uint32), sp[:s].cpu().numpy())


def check(p, dirs, d=None):
    status, ext, s, sp = run_filter(dev(p) if d is None else d, dirs)
    assert status == ch.CH_OK
    assert np.array_equal(ext, oracle.kgon_extremes(p, dirs))
    want = oracle.kgon_filter(p, dirs)
    assert np.array_equal(s, want), (len(s), len(want))
    assert np.array_equal(sp.view(np.uint32), p[want].view(np.uint32))
    return len(want)


@pytest.mark.parametrize("K", [8, 64])
@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
@pytest.mark.parametrize("n", [1, 5, 1025, 4097, 100_003, (1 << 20) + 7])
def test_filter_parity(K, dist, n):
    p = pointgen.make_points(dist, n, seed=700 + n)
    check(p, pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=K + n)))


@pytest.mark.parametrize("K", [16, 32])
@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_filter_parity_middle_k(K, dist):
    p = pointgen.make_points(dist, 300_001, seed=K)
    check(p, pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=5)))
    check(p, pointgen.kgon_directions(K))   # no offsets: axis and diagonal keys are the octagon's


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_eight_integer_directions_equal_ch_filter(dist):
    p = pointgen.make_points(dist, 500_000, seed=3)
    d = dev(p)
    ws = ch.Workspace(len(p))
    e = ch.extremes(d, ws)
    idx, sp, cnt = ch.filter_points(d, e, ws)
    s_oct = idx[: int(cnt.item())].cpu().numpy()
    status, ext, s, _ = run_filter(d, pointgen.kgon_directions(8))
    assert status == ch.CH_OK
    assert np.array_equal(ext, e.cpu().numpy().view(np.uint32))
    assert np.array_equal(s, s_oct.view(np.uint32))


def degenerate_sets():
    rng = np.random.default_rng(11)
    t = rng.uniform(-5, 5, 20000).astype(np.float32)
    g = np.array([(x, y) for x in range(-40, 41) for y in range(-40, 41)], np.float32)
    return [
        np.full((9000, 2), 0.25, np.float32),
        np.stack([t, np.float32(2) * t], 1),
        g[rng.permutation(len(g))],
        (rng.standard_normal((20000, 2)) * 1e-40).astype(np.float32),
        np.clip(rng.standard_normal((20000, 2)) * 1e37, -3e38, 3e38).astype(np.float32),
        pointgen.lattice_circle(1105),
        np.array([(1.5, -2.0), (-3.0, 7.0)], np.float32),
    ]


@pytest.mark.parametrize("K", [8, 16, 64])
@pytest.mark.parametrize("case", range(7))
def test_degenerate(K, case):
    p = degenerate_sets()[case]
    check(p, pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=case)))


@pytest.mark.parametrize("K", [16, 64])
def test_unaligned_view(K):
    p = pointgen.make_points("displaced", 200_001, seed=9)
    d = dev(np.concatenate([np.zeros((1, 2), np.float32), p]))[1:]
    assert d.data_ptr() % 16 == 8
    check(p, pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=2)), d)


@pytest.mark.parametrize("K", [8, 32, 64])
@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_hull_parity(K, dist):
    p = pointgen.make_points(dist, 400_003, seed=K)
    idx, cnt = ch.convex_hull_kgon(dev(p), pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=1)))
    torch.cuda.synchronize()
    h = idx[: int(cnt.item())].cpu().numpy().view(np.uint32)
    assert np.array_equal(h, oracle.hull(p))


def test_nonfinite_is_reported():
    p = pointgen.make_points("normal", 50_000, seed=2)
    p[777, 0] = np.inf
    status, _, s, _ = run_filter(dev(p), pointgen.kgon_directions(16))
    assert status == ch.CH_ERR_NONFINITE and len(s) == 0


def test_workspace_reuse_across_k():
    ws = ch.Workspace(200_000)
    for k, K in enumerate([64, 8, 32, 16, 64]):
        p = pointgen.make_points(pointgen.DISTRIBUTIONS[k % 3], 200_000 - 17 * k, seed=k)
        dirs = pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=k))
        status, ext, s, _ = run_filter(dev(p), dirs, ws)
        assert status == ch.CH_OK
        assert np.array_equal(ext, oracle.kgon_extremes(p, dirs))
        assert np.array_equal(s, oracle.kgon_filter(p, dirs))
