"""GPU parity of ch_hull_batched: every set's hull (set-local indices) equals
the oracle's hull of that set alone, bit for bit, for batches that mix
empty, tiny, ragged and multi-tile sets, degenerate sets and more sets than
one block of the bookkeeping kernels has threads."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_10581_gb300 as ch
import pointgen

pytestmark = pytest.mark.gpu


def run_batched(pts, offsets, ws=None):
    d = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    o = torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    ws = ws or ch.Workspace(max(len(pts), 1), num_sets=max(len(offsets) - 1, 1))
    idx, hoff = ch.convex_hull_batched(d, o, ws)
    status = ch.ch_last_error(ws.buf)
    return idx.cpu().numpy().view(np.uint32), hoff.cpu().numpy(), status


def concat(sets):
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([len(s) for s in sets])
    pts = np.concatenate(sets) if sets else np.zeros((0, 2), np.float32)
    return pts.astype(np.float32).reshape(-1, 2), offsets


def check_batch(pts, offsets, ws=None, sample=None):
    idx, hoff, status = run_batched(pts, offsets, ws)
    assert status == ch.CH_OK
    B = len(offsets) - 1
    assert hoff[0] == 0 and np.all(np.diff(hoff) >= 0)
    todo = range(B) if sample is None else sample
    for b in todo:
        p = pts[offsets[b]:offsets[b + 1]]
        got = idx[hoff[b]:hoff[b + 1]]
        want = oracle.convex_hull(p)[2] if len(p) else np.zeros(0, np.uint32)
        assert np.array_equal(got, want), (b, len(p), len(got), len(want))
    return idx, hoff


def test_mixed_sizes_and_distributions():
    sizes = [0, 1, 2, 3, 5, 63, 4095, 4096, 4097, 0, 12289, 100_003, 70_000, 8191, 1]
    sets = [pointgen.make_points(pointgen.DISTRIBUTIONS[k % 3], n, seed=300 + k) for k, n in enumerate(sizes)]
    check_batch(*concat(sets))


def test_sets_with_the_fan_test():
    # sets with at least 2^16 octagon survivors get the fan test: circle and
    # displaced-circle sets from just above that size to several refine work
    # items (64 tiles each), scaled and shifted, between small sets
    rng = np.random.default_rng(11)
    sets = []
    for k, (dist, n) in enumerate([("circle", 1_000_003), ("normal", 300), ("displaced", 500_001),
                                   ("circle", 70_000), ("displaced", 66_000), ("normal", 1_000_000),
                                   ("circle", 262_145), ("displaced", 4095), ("circle", 65_536)]):
        p = pointgen.make_points(dist, n, seed=500 + k).astype(np.float64)
        p = p * rng.uniform(0.1, 10.0) + rng.uniform(-50, 50, 2)
        sets.append(p.astype(np.float32))
    check_batch(*concat(sets))


def test_generated_batch_uneven_sizes():
    pts, offsets, _ = pointgen.make_batch(200, seed=7, min_n=100, max_n=200_000)
    check_batch(pts, offsets)


def test_many_small_sets():
    rng = np.random.default_rng(3)
    sizes = rng.integers(0, 60, 5000)
    sets = [pointgen.make_points(pointgen.DISTRIBUTIONS[k % 3], int(n), seed=k) for k, n in enumerate(sizes)]
    check_batch(*concat(sets))


def test_large_sets_with_many_super_chunks():
    sets = [pointgen.make_points("circle", (1 << 20) + 7, seed=1),
            pointgen.make_points("normal", 1000, seed=2),
            pointgen.make_points("displaced", 600_001, seed=3),
            pointgen.make_points("circle", 4097 * 3, seed=4)]
    check_batch(*concat(sets))


def degenerate_sets():
    rng = np.random.default_rng(5)
    t = rng.uniform(-5, 5, 20000).astype(np.float32)
    g = np.array([(x, y) for x in range(-40, 41) for y in range(-40, 41) if abs(x) + abs(y) <= 60], np.float32)
    sz = rng.integers(-1, 2, size=(10000, 2)).astype(np.float32)
    sz[rng.random(sz.shape) < 0.5] *= -1.0
    inner = rng.uniform(-1, 1, (30000, 2)).astype(np.float32)
    square = np.clip(np.concatenate([inner, np.array([(1, 1), (-1, 1), (-1, -1), (1, -1)], np.float32)]), -1, 1)
    base = pointgen.make_points("circle", 3000, seed=9)
    return [
        np.array([(1.5, -2.0)], np.float32),
        np.array([(1.5, -2.0), (-3.0, 7.0)], np.float32),
        np.full((9000, 2), 0.25, np.float32),
        np.stack([t, np.float32(2) * t], 1),
        g[rng.permutation(len(g))],
        sz,
        (rng.standard_normal((20000, 2)) * 1e-40).astype(np.float32),
        np.clip(rng.standard_normal((20000, 2)) * 1e38, -3.4e38, 3.4e38).astype(np.float32),
        square.astype(np.float32),
        base[rng.integers(0, 3000, 50000)],
        np.stack([np.zeros(5000, np.float32), rng.standard_normal(5000).astype(np.float32)], 1),
    ]


def test_degenerate_sets():
    check_batch(*concat(degenerate_sets()))


def test_single_set_matches_ch_hull():
    p = pointgen.make_points("displaced", 300_000, seed=11)
    idx, hoff = check_batch(*concat([p]))
    hidx, hcnt = ch.convex_hull(torch.from_numpy(p).cuda())
    h = int(hcnt.item())
    assert hoff[1] == h
    assert np.array_equal(idx[:h], hidx[:h].cpu().numpy().view(np.uint32))


def test_zero_sets():
    d = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    o = torch.zeros(1, dtype=torch.int64, device="cuda")
    idx, hoff = ch.convex_hull_batched(d, o, ch.Workspace(1))
    assert hoff.cpu().tolist() == [0]


def test_workspace_reuse():
    ws = ch.Workspace(400_000, num_sets=300)
    for k in range(3):
        pts, offsets, _ = pointgen.make_batch(100 + 100 * k, seed=20 + k, min_n=10, max_n=5000)
        assert offsets[-1] <= 400_000
        check_batch(pts, offsets, ws)


@pytest.mark.parametrize("bad", ["first_not_zero", "decreasing", "negative"])
def test_malformed_offsets_are_argument_errors(bad):
    pts, offsets = concat([pointgen.make_points("normal", 5000, seed=k) for k in range(4)])
    ws = ch.Workspace(len(pts), num_sets=4)
    o = offsets.copy()
    if bad == "first_not_zero":
        o[0] = 1
    elif bad == "decreasing":
        o[2] = o[1] - 1
    else:
        o[1] = -5
    _, hoff, status = run_batched(pts, o, ws)
    assert status == ch.CH_ERR_ARG
    assert np.all(hoff == 0)
    check_batch(pts, offsets, ws)   # the workspace stays usable


def test_points_beyond_the_workspace_are_a_capacity_error():
    pts, offsets = concat([pointgen.make_points("normal", 5000, seed=k) for k in range(4)])
    ws = ch.Workspace(1000, num_sets=4)
    _, hoff, status = run_batched(pts, offsets, ws)
    assert status == ch.CH_ERR_CAPACITY
    assert np.all(hoff == 0)


def test_nonfinite_set_gets_an_empty_hull_and_the_others_are_exact():
    sets = [pointgen.make_points("normal", 20000, seed=k) for k in range(5)]
    sets[2][777, 1] = np.inf
    pts, offsets = concat(sets)
    idx, hoff, status = run_batched(pts, offsets)
    assert status == ch.CH_ERR_NONFINITE
    assert hoff[3] == hoff[2]
    for b in (0, 1, 3, 4):
        want = oracle.convex_hull(sets[b])[2]
        assert np.array_equal(idx[hoff[b]:hoff[b + 1]], want)


def test_cuda_graph_replay():
    """The batched call captures into a CUDA graph (no allocation, no host
    synchronisation); replays read the current contents of the buffers."""
    pts, offsets, _ = pointgen.make_batch(64, seed=31, min_n=50, max_n=20_000)
    d = torch.from_numpy(pts).cuda()
    o = torch.from_numpy(offsets).cuda()
    ws = ch.Workspace(len(pts), num_sets=64)
    idx = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    hoff = torch.zeros(65, dtype=torch.int64, device="cuda")
    ch.ch_hull_batched(d, o, idx, hoff, ws.buf)   # first call outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ch.ch_hull_batched(d, o, idx, hoff, ws.buf)
    for seed in (31, 32):
        p2, off2, _ = pointgen.make_batch(64, seed=31, min_n=50, max_n=20_000)
        if seed == 32:   # same set sizes, new coordinates
            p2 = (p2 * np.float32(-1.5)).astype(np.float32)
        d.copy_(torch.from_numpy(p2))
        graph.replay()
        torch.cuda.synchronize()
        assert ch.ch_last_error(ws.buf) == ch.CH_OK
        h = hoff.cpu().numpy()
        got = idx.cpu().numpy().view(np.uint32)
        for b in range(64):
            want = oracle.convex_hull(p2[offsets[b]:offsets[b + 1]])[2]
            assert np.array_equal(got[h[b]:h[b + 1]], want), (seed, b)


GRID_KNOBS = ("bx_extremes", "bx_filter", "bx_sort_pass", "bx_emit")


@pytest.mark.parametrize("per_sm,stride,chunk,items", [(1, 1, 8, 4), (3, 3, 16, 8), (16, 4, 64, 16)])
def test_launch_shapes_do_not_change_results(per_sm, stride, chunk, items):
    """Every batched kernel walks tiles grid-stride, by ticket or over its
    own range, and the fan's vertices are input points whatever tiles the
    bins sample: any grid, sampling stride, work-item size and points per
    thread give the same hulls (the batch has sets with the fan)."""
    pts, offsets, _ = pointgen.make_batch(300, seed=41, min_n=50, max_n=300_000)
    extra = pointgen.make_points("circle", 400_000, seed=42)   # several fan work items
    pts = np.concatenate([pts, extra])
    offsets = np.concatenate([offsets, [offsets[-1] + len(extra)]])
    try:
        for k in GRID_KNOBS:
            ch.ch_tune_set(k, per_sm)
        ch.ch_tune_set("bx_fan_stride", stride)
        ch.ch_tune_set("bx_fan_chunk", chunk)
        ch.ch_tune_set("bx_ext_items", items)
        check_batch(pts, offsets, sample=list(range(0, 300, 7)) + [300])
    finally:
        for k in ch.TUNE_KNOBS:
            ch.ch_tune_set(k, 0)


def test_autotuner_keeps_results_and_caches(tmp_path):
    from paper_2303_10581_gb300 import autotune
    pts, offsets, _ = pointgen.make_batch(128, seed=43, min_n=100, max_n=100_000)
    d, o = torch.from_numpy(pts).cuda(), torch.from_numpy(offsets).cuda()
    ws = ch.Workspace(len(pts), num_sets=128)
    try:
        res = autotune.tune(d, o, ws, reps=1)
        assert res["ms_best"] <= res["ms_default"]
        assert autotune.current() == res["config"]
        path = str(tmp_path / "tune.json")
        key = autotune.cache_key(d.device, 128, len(pts))
        autotune.save(res, key, path)
        assert autotune.load_cached(key, path) == res
        check_batch(pts, offsets, ws, sample=range(0, 128, 5))
    finally:
        autotune.apply({})
