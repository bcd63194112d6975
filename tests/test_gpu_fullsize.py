"""Full-size parity: the single-set workloads at n = 10^8 (three
distributions) and intermediate sizes, whole survivor and hull lists
against the oracle, with the same launch configuration the benchmark uses
(ch_hull on one set, workspace sized for the set)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _gpu_path(p):
    d = torch.from_numpy(p).cuda()
    n = len(p)
    ws = ch.Workspace(n)
    ext = ch.extremes(d, ws)
    idx, _, cnt = ch.filter_points(d, ext, ws, with_points=False)
    hidx, hcnt = ch.convex_hull(d, ws)
    ws.check()
    s, h = int(cnt.item()), int(hcnt.item())
    out = (ext.cpu().numpy().view(np.uint32), idx[:s].cpu().numpy().view(np.uint32),
           hidx[:h].cpu().numpy().view(np.uint32))
    del d, ws, idx, hidx
    torch.cuda.empty_cache()
    return out


def _compare(p):
    e, s, h = _gpu_path(p)
    oe = oracle.extremes(p)
    assert np.array_equal(e, oe)
    os_ = oracle.filter_points(p, oe)
    assert len(s) == len(os_)
    assert np.array_equal(s, os_)
    oh = oracle.hull(p, os_)
    assert len(h) == len(oh), (len(h), len(oh))
    assert np.array_equal(h, oh)


@pytest.mark.parametrize("n", [4_000_037, 16_000_057])
@pytest.mark.parametrize("dist", ["circle", "displaced"])
def test_dense_sets(dist, n):
    _compare(pointgen.make_points(dist, n, seed=n % 97))


def _structured(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "parabola":            # every point on a convex curve: huge lower chain
        x = rng.uniform(-1, 1, n)
        return np.stack([x, x * x], 1).astype(np.float32)
    if kind == "two_parabolas":       # a lens: long lower and upper chains
        x = rng.uniform(-1, 1, n)
        y = np.where(rng.random(n) < 0.5, x * x - 1, 1 - x * x)
        return np.stack([x, y], 1).astype(np.float32)
    if kind == "clusters":            # Gaussian blobs of very different scales: long bridges
        k = 16
        centres = rng.uniform(-100, 100, (k, 2))
        scales = np.exp(rng.uniform(np.log(1e-3), np.log(10), k))
        lab = rng.integers(0, k, n)
        return (centres[lab] + rng.standard_normal((n, 2)) * scales[lab, None]).astype(np.float32)
    if kind == "grid_ring":           # integer ring: many ties, collinear runs, duplicates
        r = rng.integers(900, 1001, n)
        th = rng.uniform(0, 2 * np.pi, n)
        return np.stack([np.round(r * np.cos(th)), np.round(r * np.sin(th))], 1).astype(np.float32)
    raise ValueError(kind)


def test_workspace_reuse_across_large_sets():
    """One workspace, several calls whose chain compaction spans several
    look-back tiles: nothing a call leaves behind may change the next."""
    n = 3_000_000
    ws = ch.Workspace(n)
    for k, dist in enumerate(["circle", "normal", "displaced", "circle"]):
        p = pointgen.make_points(dist, n - 1000 * k, seed=50 + k)
        d = torch.from_numpy(p).cuda()
        hidx, hcnt = ch.convex_hull(d, ws)
        ws.check()
        h = int(hcnt.item())
        assert np.array_equal(hidx[:h].cpu().numpy().view(np.uint32), oracle.hull(p)), (k, dist)


@pytest.mark.parametrize("kind", ["parabola", "two_parabolas", "clusters", "grid_ring"])
def test_structured_sets(kind):
    _compare(_structured(kind, 3_000_017, seed=7))


@pytest.mark.parametrize("k,dist", list(enumerate(pointgen.DISTRIBUTIONS)))
def test_bench_workload_1e8(k, dist):
    # the benchmark's inputs: seed 1 + position of the distribution
    _compare(pointgen.make_points(dist, 100_000_000, seed=1 + k))
