"""GPU parity of the hull with a second polygon over the octagon's
survivors (ch_hull_octagon_kgon) and of the learned proposal run end to end
on the device (ch_hull_learned): the hull equals the oracle's, bit for bit;
the second polygon's vertices are, for every direction, the octagon
survivor with the largest key (lowest index on ties), checked against the
oracle's K-direction extremes over the oracle's octagon survivors."""
import numpy as np
import pytest
import torch

import oracle
import oracle_par
import paper_2303_10581_gb300 as ch
import pointgen
from paper_2303_10581_gb300 import learned

pytestmark = pytest.mark.gpu


def run(p, K, dirs, offset=False):
    big = torch.from_numpy(np.concatenate([np.zeros((1, 2), np.float32), p])).cuda()
    d = big[1:] if offset else big[1:].clone()
    n = len(p)
    ws = ch.Workspace(n)
    ext = torch.full((K,), -1, dtype=torch.int32, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dd = torch.from_numpy(np.ascontiguousarray(dirs, np.float32)).cuda()
    ch.ch_hull_octagon_kgon(d, dd, K, ext, idx, cnt, ws.buf)
    ws.check()
    spec = ch.ch_hull_counts(ws.buf, n)[2]
    return idx[: int(cnt.item())].cpu().numpy().view(np.uint32), ext.cpu().numpy().view(np.uint32), spec


def survivor_extremes(p, dirs):
    s1 = oracle_par.filter_points(p, oracle.extremes(p))
    return s1[oracle.kgon_extremes(p[s1], dirs)], s1


CASES = [("normal", 100_003), ("circle", 100_003), ("displaced", 300_007), ("gaussians", 1_000_003),
         ("ellipse", 1_000_003), ("displaced", 4097)]


@pytest.mark.parametrize("K", [8, 16, 32, 64])
@pytest.mark.parametrize("kind,n", CASES)
def test_hull_and_vertices(kind, n, K):
    seed = 70 + n % 97 + K
    p = (pointgen.make_points(kind, n, seed=seed) if kind in pointgen.DISTRIBUTIONS
         else pointgen.make_family(kind, n, seed=seed))
    dirs = pointgen.kgon_directions(K, pointgen.kgon_offsets(K, seed=K + 1) if K > 8 else None)
    h, ext, spec = run(p, K, dirs)
    assert np.array_equal(h, oracle.convex_hull(p)[2])
    if K > 8 and not spec:
        want, _ = survivor_extremes(p, dirs)
        assert np.array_equal(ext, want)


def test_unaligned_view():
    p = pointgen.make_family("ellipse", 500_001, seed=5)
    dirs = pointgen.kgon_directions(32, pointgen.kgon_offsets(32, seed=9))
    h, ext, spec = run(p, 32, dirs, offset=True)
    assert np.array_equal(h, oracle.convex_hull(p)[2])
    want, _ = survivor_extremes(p, dirs)
    assert spec == 0 and np.array_equal(ext, want)


def test_large_normal_set_with_the_speculative_sweep():
    # the speculative sweep serves the filter: no keep bits, the second
    # polygon does not run, the hull is the same
    p = pointgen.make_points("normal", (1 << 22) + 13, seed=1)
    dirs = pointgen.kgon_directions(16)
    h, _, spec = run(p, 16, dirs)
    assert spec == 1
    assert np.array_equal(h, oracle_par.hull(p, oracle_par.filter_points(p, oracle.extremes(p))))


def test_degenerate_sets():
    rng = np.random.default_rng(2)
    for p in (np.zeros((5000, 2), np.float32), np.stack([np.arange(7000.0), np.arange(7000.0)], 1).astype(np.float32),
              rng.integers(-3, 4, (20000, 2)).astype(np.float32)):
        dirs = pointgen.kgon_directions(64, pointgen.kgon_offsets(64, seed=3))
        h, _, _ = run(p, 64, dirs)
        assert np.array_equal(h, oracle.convex_hull(p)[2])


@pytest.mark.parametrize("kind", pointgen.FAMILIES)
def test_learned_end_to_end_on_the_device(kind):
    """Whatever the (untrained) MLP picks, the hull is the oracle's; the
    choice comes back through k_out and dirs_out."""
    p = pointgen.make_family(kind, 600_011, seed=13)
    d = torch.from_numpy(p).cuda()
    ws = ch.Workspace(len(p))
    for seed in (1, 2, 3):
        prop = learned.Proposal(seed=seed)
        hidx, hcnt, K, dirs = prop.hull_on_device(d, ws)
        ws.check()
        assert K in (8, 16, 32, 64)
        assert np.all(np.abs(dirs[:K]) <= 1.0) and np.all(dirs[K:] == 0.0)
        assert np.array_equal(hidx[: int(hcnt.item())].cpu().numpy().view(np.uint32), oracle.convex_hull(p)[2])
