"""Autotuner of ch_hull_batched's launch shapes.

A coordinate search over the launch knobs (``ch_tune_set``: blocks per SM
of four kernels, the tile sampling and work-item size of the fan, the
points per thread and block size of the extremes sweep) on a given batch, timing the batched call with CUDA events; the best setting is
cached in a JSON file keyed by the GPU and the batch's shape (sets and
points, rounded to powers of two) and applied with ``apply``.  Results of
the call do not depend on the knobs, only its speed.
"""
from __future__ import annotations

import json
import math
import os

from . import TUNE_KNOBS, ch_hull_batched, ch_tune_get, ch_tune_set

CANDIDATES = {
    "bx_extremes": (2, 4, 8, 16),      # blocks per SM
    "bx_filter": (2, 4, 6, 8),
    "bx_sort_pass": (1, 2, 3),
    "bx_emit": (1, 2, 4, 8),
    "bx_fan_stride": (1, 2, 4),        # the fan's bins sample every k-th tile
    "bx_fan_chunk": (16, 32, 64),      # tiles per work item of the fan refine
    "bx_ext_items": (4, 8, 16),        # points per thread per tile (block of 1024, 512, 256 threads)
}
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "convhull_gb300", "tune.json")


def cache_key(device, num_sets: int, n: int) -> str:
    import torch
    prop = torch.cuda.get_device_properties(device)
    b = lambda v: 1 << max(0, round(math.log2(max(v, 1))))
    return f"{prop.name}|sms={prop.multi_processor_count}|sets~{b(num_sets)}|points~{b(n)}"


def current() -> dict:
    return {k: ch_tune_get(k) for k in TUNE_KNOBS}


def apply(config: dict) -> None:
    for k in TUNE_KNOBS:
        ch_tune_set(k, int(config.get(k, 0)))


def time_batched(pts, offsets, idx, hoff, ws, reps: int = 3) -> float:
    import torch
    ch_hull_batched(pts, offsets, idx, hoff, ws.buf)      # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ch_hull_batched(pts, offsets, idx, hoff, ws.buf)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(pts, offsets, ws, reps: int = 3, rounds: int = 1) -> dict:
    """Coordinate search from the built-in choice; leaves the best setting
    applied and returns it with the default and best times (ms)."""
    import torch
    n = pts.shape[0]
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    hoff = torch.zeros(offsets.shape[0], dtype=torch.int64, device=pts.device)
    best = {k: 0 for k in TUNE_KNOBS}
    apply(best)
    best_ms = t_default = time_batched(pts, offsets, idx, hoff, ws, reps)
    for _ in range(rounds):
        for k in TUNE_KNOBS:
            for v in CANDIDATES.get(k, ()):   # (knobs of the single-set call are not the batch's)
                trial = dict(best, **{k: v})
                apply(trial)
                t = time_batched(pts, offsets, idx, hoff, ws, reps)
                if t < best_ms:
                    best, best_ms = trial, t
    apply(best)
    return {"config": best, "ms_default": round(t_default, 4), "ms_best": round(best_ms, 4)}


def save(result: dict, key: str, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    data = json.load(open(path)) if os.path.exists(path) else {}
    data[key] = result
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=2)
    os.replace(tmp, path)


def load_cached(key: str, path: str = DEFAULT_CACHE):
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(key)
