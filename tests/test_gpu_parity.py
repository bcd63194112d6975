"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, on seeded inputs that span several tiles with ragged
tails, plus the degenerate cases.  Survivor lists and hull lists must be
bit-exact (they are index lists)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 63, 64, 65, 4095, 4096, 4097, 12289, 100_003, (1 << 20) + 7]


def dev(p):
    return torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()


def gpu_all(p, ws=None):
    """extremes, survivors (idx, pts), hull via the three entry points."""
    d = dev(p)
    n = len(p)
    ws = ws or ch.Workspace(max(n, 1))
    e = ch.extremes(d, ws)
    idx, sp, cnt = ch.filter_points(d, e, ws)
    hidx, hcnt = ch.convex_hull(d, ws)
    torch.cuda.synchronize()
    assert ch.ch_last_error(ws.buf) == ch.CH_OK
    s = int(cnt.item())
    h = int(hcnt.item())
    return (e.cpu().numpy().view(np.uint32), idx[:s].cpu().numpy().view(np.uint32),
            sp[:s].cpu().numpy(), hidx[:h].cpu().numpy().view(np.uint32))


def check_against_oracle(p, ws=None):
    e, s, spts, h = gpu_all(p, ws)
    oe, os_, oh = oracle.convex_hull(p)
    assert np.array_equal(e, oe), (e, oe)
    assert np.array_equal(s, os_), (len(s), len(os_))
    assert np.array_equal(spts.view(np.uint32), p[os_].view(np.uint32))
    assert np.array_equal(h, oh), (len(h), len(oh))
    return len(s), len(h)


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
@pytest.mark.parametrize("n", SIZES)
def test_parity_sizes(dist, n):
    p = pointgen.make_points(dist, n, seed=1000 + n)
    check_against_oracle(p)


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
def test_parity_unaligned_points(dist):
    # a view starting one point in: 8-byte but not 16-byte aligned
    p = pointgen.make_points(dist, 50_001, seed=77)
    big = dev(np.concatenate([np.zeros((1, 2), np.float32), p]))
    d = big[1:]
    assert d.data_ptr() % 16 == 8
    ws = ch.Workspace(len(p))
    e = ch.extremes(d, ws)
    idx, sp, cnt = ch.filter_points(d, e, ws)
    hidx, hcnt = ch.convex_hull(d, ws)
    oe, os_, oh = oracle.convex_hull(p)
    assert np.array_equal(e.cpu().numpy().view(np.uint32), oe)
    s = int(cnt.item())
    assert np.array_equal(idx[:s].cpu().numpy().view(np.uint32), os_)
    assert np.array_equal(hidx[: int(hcnt.item())].cpu().numpy().view(np.uint32), oh)


def test_workspace_reuse_across_sizes_and_distributions():
    ws = ch.Workspace(300_000)
    for k, dist in enumerate(["circle", "normal", "displaced", "circle", "normal"]):
        p = pointgen.make_points(dist, 300_000 - 37 * k, seed=k)
        check_against_oracle(p, ws)


def test_empty_input():
    ws = ch.Workspace(1)
    d = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    ext = torch.zeros(8, dtype=torch.int32, device="cuda")
    idx, sp, cnt = ch.filter_points(d, ext, ws)
    hidx, hcnt = ch.convex_hull(d, ws)
    assert int(cnt.item()) == 0 and int(hcnt.item()) == 0


@pytest.mark.parametrize("case", [
    "single", "pair", "all_equal", "collinear", "grid", "signed_zero", "subnormal", "huge", "square",
    "lattice", "duplicates", "vertical_line",
])
def test_degenerate_cases(case):
    rng = np.random.default_rng(5)
    if case == "single":
        p = np.array([(1.5, -2.0)], np.float32)
    elif case == "pair":
        p = np.array([(1.5, -2.0), (-3.0, 7.0)], np.float32)
    elif case == "all_equal":
        p = np.full((9000, 2), 0.25, np.float32)
    elif case == "collinear":
        t = rng.uniform(-5, 5, 20000).astype(np.float32)
        p = np.stack([t, np.float32(2) * t], 1)
    elif case == "grid":
        g = np.array([(x, y) for x in range(-40, 41) for y in range(-40, 41) if abs(x) + abs(y) <= 60], np.float32)
        p = g[rng.permutation(len(g))]
    elif case == "signed_zero":
        p = rng.integers(-1, 2, size=(10000, 2)).astype(np.float32)
        p[rng.random(p.shape) < 0.5] *= -1.0   # makes -0.0 entries
    elif case == "subnormal":
        p = (rng.standard_normal((20000, 2)) * 1e-40).astype(np.float32)
    elif case == "huge":
        p = (rng.standard_normal((20000, 2)) * 1e38).astype(np.float32)
        p = np.clip(p, -3.4e38, 3.4e38).astype(np.float32)
    elif case == "square":
        inner = rng.uniform(-1, 1, (30000, 2)).astype(np.float32)
        p = np.concatenate([inner, np.array([(1, 1), (-1, 1), (-1, -1), (1, -1)], np.float32)])
        p = np.clip(p, -1, 1)
    elif case == "lattice":
        p = pointgen.lattice_circle(1185665)
        p = p[rng.permutation(len(p))]
    elif case == "duplicates":
        base = pointgen.make_points("circle", 3000, seed=9)
        p = base[rng.integers(0, 3000, 50000)]
    else:
        p = np.stack([np.zeros(5000, np.float32), rng.standard_normal(5000).astype(np.float32)], 1)
    check_against_oracle(p)


def test_near_edge_points_take_the_exact_paths():
    """Points placed on and one ulp around the polygon's edges: the binary32
    test cannot decide them, so the binary64 and expansion tiers must."""
    rng = np.random.default_rng(17)
    base = pointgen.make_points("normal", 40_000, seed=3)
    e = oracle.extremes(base)
    v = base[e]
    extra = []
    for k in range(8):
        a, b = v[k].astype(np.float64), v[(k + 1) % 8].astype(np.float64)
        for t in rng.uniform(0, 1, 400):
            q = (a + t * (b - a)).astype(np.float32)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    r = q.copy()
                    if dx:
                        r[0] = np.nextafter(r[0], np.float32(dx * np.inf))
                    if dy:
                        r[1] = np.nextafter(r[1], np.float32(dy * np.inf))
                    extra.append(r)
    p = np.concatenate([base, np.array(extra, np.float32)])
    s, h = check_against_oracle(p)
    assert s > 1000   # plenty of the near-edge points survive


def test_filter_with_oracle_extremes():
    p = pointgen.make_points("displaced", 200_000, seed=12)
    oe = oracle.extremes(p)
    d = dev(p)
    ext = torch.from_numpy(oe.view(np.int32)).cuda()
    idx, sp, cnt = ch.filter_points(d, ext, ch.Workspace(len(p)))
    s = int(cnt.item())
    assert np.array_equal(idx[:s].cpu().numpy().view(np.uint32), oracle.filter_points(p, oe))


def test_nonfinite_is_reported():
    p = pointgen.make_points("normal", 10000, seed=2)
    p[4321, 0] = np.nan
    ws = ch.Workspace(len(p))
    d = dev(p)
    ch.extremes(d, ws)
    assert ch.ch_last_error(ws.buf) == ch.CH_ERR_NONFINITE
    hidx, hcnt = ch.convex_hull(d, ws)
    assert ch.ch_last_error(ws.buf) == ch.CH_ERR_NONFINITE
    assert int(hcnt.item()) == 0
    assert ch.ch_last_error(ws.buf) == ch.CH_OK
    # the workspace stays usable
    q = pointgen.make_points("normal", 10000, seed=3)
    check_against_oracle(q, ws)


def test_out_of_range_extreme_index_is_an_argument_error():
    p = pointgen.make_points("normal", 1000, seed=2)
    ws = ch.Workspace(len(p))
    ext = torch.tensor([0, 1, 2, 3, 4, 5, 6, 5000], dtype=torch.int32, device="cuda")
    idx, sp, cnt = ch.filter_points(dev(p), ext, ws)
    assert ch.ch_last_error(ws.buf) == ch.CH_ERR_ARG
    assert int(cnt.item()) == 0


@pytest.mark.parametrize("dist", pointgen.DISTRIBUTIONS)
@pytest.mark.parametrize("n", [4095, 100_003, (1 << 20) + 7])
def test_parity_single_pass_variant(dist, n):
    """The single-pass look-back compaction gives the same lists."""
    ch.ch_filter_variant(1)
    try:
        check_against_oracle(pointgen.make_points(dist, n, seed=2000 + n))
    finally:
        ch.ch_filter_variant(0)


def test_filter_variant_rejects_unknown():
    with pytest.raises(ch.CHError):
        ch.ch_filter_variant(7)


def _kgon_case(case, rng):
    if case == "displaced_ellipse":
        p = pointgen.make_points("displaced", 300_000, seed=41).astype(np.float64)
        p[:, 0] *= 10.0
        return p.astype(np.float32)
    if case == "ring_outliers":
        p = pointgen.make_points("displaced", 250_000, seed=42)
        far = (rng.standard_normal((50, 2)) * 3).astype(np.float32)
        return np.concatenate([p, far])
    if case == "collinear_big":
        t = rng.uniform(-5, 5, 200_000).astype(np.float32)
        return np.stack([t, np.float32(3) * t + np.float32(1)], 1)
    if case == "duplicated_ring":
        base = pointgen.make_points("displaced", 5_000, seed=43)
        return base[rng.integers(0, 5_000, 300_000)]
    if case == "square_boundary":
        t = rng.uniform(-1, 1, 300_000).astype(np.float32)
        side = rng.integers(0, 4, 300_000)
        one = np.ones_like(t)
        x = np.where(side == 0, one, np.where(side == 1, -one, t))
        y = np.where(side == 2, one, np.where(side == 3, -one, t))
        return np.stack([x, y], 1).astype(np.float32)
    if case == "tiny_scale":
        return (pointgen.make_points("displaced", 200_000, seed=44) * np.float32(1e-30)).astype(np.float32)
    if case == "huge_scale":
        return (pointgen.make_points("displaced", 200_000, seed=45) * np.float32(1e30)).astype(np.float32)
    if case == "four_wedges":   # most fan bins see no sample point
        th = rng.uniform(-0.05, 0.05, 300_000) + rng.integers(0, 4, 300_000) * (np.pi / 2)
        r = 1.0 - np.abs(rng.standard_normal(300_000)) * 0.01
        return np.stack([r * np.cos(th), r * np.sin(th)], 1).astype(np.float32)
    if case == "half_ring":
        th = rng.uniform(0.0, np.pi, 300_000)
        return np.stack([np.cos(th), np.sin(th)], 1).astype(np.float32)
    raise ValueError(case)


@pytest.mark.parametrize("case", ["displaced_ellipse", "ring_outliers", "collinear_big", "duplicated_ring",
                                  "square_boundary", "tiny_scale", "huge_scale", "four_wedges", "half_ring"])
def test_second_polygon_cases(case):
    """Inputs with at least 2^16 octagon survivors, so the hull step's fan
    (vertices: the farthest sampled points of angular bins around the
    bounding-box centre) is built and, where it removes enough, applied --
    including fans with flat or clockwise triangles, bins without samples,
    points on fan edges and extreme scales."""
    p = _kgon_case(case, np.random.default_rng(7))
    check_against_oracle(p)


@pytest.mark.parametrize("dist", ["circle", "displaced"])
@pytest.mark.parametrize("aligned", [True, False])
def test_fan_removes_points_and_keeps_the_hull(dist, aligned):
    """On circle-like sets the fan drops octagon survivors before the sort
    (fewer points sorted than survived the octagon), for 16-byte-aligned
    point pairs and for an 8-byte-aligned view (the two refine kernels), and
    the hull is still the oracle's."""
    p = pointgen.make_points(dist, 1_000_003, seed=91)
    if aligned:
        d = dev(p)
    else:
        d = dev(np.concatenate([np.zeros((1, 2), np.float32), p]))[1:]
        assert d.data_ptr() % 16 == 8
    ws = ch.Workspace(len(p))
    hidx, hcnt = ch.convex_hull(d, ws)
    torch.cuda.synchronize()
    assert ch.ch_last_error(ws.buf) == ch.CH_OK
    s_oct, t, _, _ = ch.ch_hull_counts(ws.buf, len(p))
    _, os_, oh = oracle.convex_hull(p)
    assert s_oct == len(os_)
    assert t < (s_oct if dist == "circle" else s_oct // 4), (s_oct, t)
    assert np.array_equal(hidx[: int(hcnt.item())].cpu().numpy().view(np.uint32), oh)
