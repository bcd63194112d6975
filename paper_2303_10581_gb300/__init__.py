"""GB300 octagon-filter convex hull (Carrasco et al., arXiv 2303.10581).

Thin ctypes binding over the C ABI in ``include/convhull.h``.  Every function
here only marshals arguments (torch tensors -> device pointers, the current
CUDA stream) and checks the returned status; all of the path's arithmetic
runs in the CUDA kernels of ``_lib/libconvhull.so``.  There is no CPU
fallback: if the library cannot be loaded, or a tensor is not on a CUDA
device, the call raises.

Low-level names mirror the C ABI (``ch_extremes``, ``ch_filter``, ``ch_extremes_filter``,
``ch_hull``, ``ch_hull_batched``, ``ch_workspace_size``,
``ch_workspace_init``, ``ch_last_error``); ``Workspace``, ``extremes``,
``filter_points`` and ``convex_hull`` are conveniences built on them.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

STATUS = {
    0: "CH_OK",
    1: "CH_ERR_ARG",
    2: "CH_ERR_NONFINITE",
    3: "CH_ERR_CAPACITY",
    4: "CH_ERR_CUDA",
    5: "CH_ERR_TIMEOUT",
    6: "CH_ERR_UNSUPPORTED",
}
CH_OK, CH_ERR_ARG, CH_ERR_NONFINITE, CH_ERR_CAPACITY, CH_ERR_CUDA, CH_ERR_TIMEOUT, CH_ERR_UNSUPPORTED = range(7)

SYMBOLS = ("ch_workspace_size", "ch_workspace_init", "ch_extremes", "ch_filter", "ch_extremes_filter", "ch_hull",
           "ch_hull_batched", "ch_last_error", "ch_probe_start", "ch_probe_stop", "ch_filter_noalloc",
           "ch_filter_variant", "ch_hull_counts", "ch_filter_kgon", "ch_hull_kgon", "ch_kgon_features",
           "ch_mlp_forward", "ch_mlp_train_step", "ch_mlp_param_count", "ch_mlp_scratch_floats",
           "ch_tune_set", "ch_tune_get", "ch_hull_octagon_kgon", "ch_hull_learned")
TUNE_KNOBS = ("bx_extremes", "bx_filter", "bx_sort_pass", "bx_emit", "bx_fan_stride", "bx_fan_chunk", "bx_ext_items",
              "fan2_min_log2")
# ch_filter_noalloc reports a device-side error as this bit | the status code in its count
NOALLOC_FAILED = 0x80000000
KERNELS = ("extremes", "octagon", "filter", "sort_hist", "sort_pass", "chain", "emit", "finish", "kgon")


class CHError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raise if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    if not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing or stale; run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    sz = ctypes.c_size_t
    lib.ch_workspace_size.argtypes = [i64, i64, ctypes.POINTER(sz)]
    lib.ch_workspace_init.argtypes = [p, sz, p]
    lib.ch_extremes.argtypes = [p, i64, p, p, sz, p]
    lib.ch_filter.argtypes = [p, i64, p, p, p, p, p, sz, p]
    lib.ch_extremes_filter.argtypes = [p, i64, p, p, p, p, p, sz, p]
    lib.ch_hull.argtypes = [p, i64, p, p, p, sz, p]
    lib.ch_hull_batched.argtypes = [p, p, ctypes.c_int32, p, p, p, sz, p]
    lib.ch_last_error.argtypes = [p, p]
    lib.ch_probe_start.argtypes = [ctypes.c_uint32, ctypes.c_int32]
    lib.ch_probe_stop.argtypes = [p, p]
    lib.ch_filter_noalloc.argtypes = [p, i64, p, p, p, p, p]
    lib.ch_filter_variant.argtypes = [ctypes.c_int32]
    lib.ch_hull_octagon_kgon.argtypes = [p, i64, p, ctypes.c_int32, p, p, p, p, sz, p]
    lib.ch_hull_learned.argtypes = [p, i64, p, p, p, p, p, p, sz, p]
    lib.ch_hull_counts.argtypes = [p, sz, i64, p, p]
    lib.ch_filter_kgon.argtypes = [p, i64, p, ctypes.c_int32, p, p, p, p, p, sz, p]
    lib.ch_hull_kgon.argtypes = [p, i64, p, ctypes.c_int32, p, p, p, sz, p]
    f32 = ctypes.c_float
    i32 = ctypes.c_int32
    lib.ch_kgon_features.argtypes = [p, i64, p, p]
    lib.ch_mlp_forward.argtypes = [p, i32, p, p, p, p, p]
    lib.ch_mlp_train_step.argtypes = [p, i32, p, p, p, f32, p, p, p, p, i32, f32, p, p, p]
    lib.ch_mlp_param_count.argtypes = []
    lib.ch_mlp_scratch_floats.argtypes = [i32]
    lib.ch_tune_set.argtypes = [i32, i32]
    lib.ch_tune_get.argtypes = [i32, ctypes.POINTER(i32)]
    for name in SYMBOLS:
        getattr(lib, name).restype = ctypes.c_int
    lib.ch_mlp_scratch_floats.restype = ctypes.c_int64
    _lib = lib
    return lib


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t, what, cuda=True):
    if t is None:
        return None
    if cuda and not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def _check(rc: int, what: str):
    if rc != CH_OK:
        raise CHError(rc, what)


# ---------------------------------------------------------------- C-ABI names

def ch_workspace_size(n: int, num_sets: int = 1) -> int:
    out = ctypes.c_size_t(0)
    _check(load().ch_workspace_size(int(n), int(num_sets), ctypes.byref(out)), "ch_workspace_size")
    return int(out.value)


def ch_workspace_init(ws, stream=None):
    _check(load().ch_workspace_init(_ptr(ws, "ws"), ws.numel() * ws.element_size(), _stream(stream)),
           "ch_workspace_init")


def ch_extremes(pts, ext8, ws, stream=None):
    _check(load().ch_extremes(_ptr(pts, "pts"), pts.shape[0], _ptr(ext8, "ext8"), _ptr(ws, "ws"),
                              ws.numel(), _stream(stream)), "ch_extremes")


def ch_filter(pts, ext8, surv_idx, surv_pts, surv_count, ws, stream=None):
    _check(load().ch_filter(_ptr(pts, "pts"), pts.shape[0], _ptr(ext8, "ext8"), _ptr(surv_idx, "surv_idx"),
                            _ptr(surv_pts, "surv_pts"), _ptr(surv_count, "surv_count"), _ptr(ws, "ws"),
                            ws.numel(), _stream(stream)), "ch_filter")


def ch_extremes_filter(pts, ext8, surv_idx, surv_pts, surv_count, ws, stream=None):
    """ch_extremes + ch_filter in one call (the speculative single sweep on
    large sets); ext8 is an output here."""
    _check(load().ch_extremes_filter(_ptr(pts, "pts"), pts.shape[0], _ptr(ext8, "ext8"), _ptr(surv_idx, "surv_idx"),
                                     _ptr(surv_pts, "surv_pts"), _ptr(surv_count, "surv_count"), _ptr(ws, "ws"),
                                     ws.numel(), _stream(stream)), "ch_extremes_filter")


def ch_filter_noalloc(pts, ext8, surv_idx, surv_pts, surv_count, stream=None):
    """ch_filter without a workspace, for callers that cannot allocate device
    memory (the library's own static scratch is used; n <= 2^26; calls that
    overlap on the GPU race).  A device-side error comes back in the count:
    0x80000000 | code (see NOALLOC_FAILED)."""
    _check(load().ch_filter_noalloc(_ptr(pts, "pts"), pts.shape[0], _ptr(ext8, "ext8"),
                                    _ptr(surv_idx, "surv_idx"), _ptr(surv_pts, "surv_pts"),
                                    _ptr(surv_count, "surv_count"), _stream(stream)), "ch_filter_noalloc")


def ch_hull(pts, hull_idx, hull_count, ws, stream=None):
    _check(load().ch_hull(_ptr(pts, "pts"), pts.shape[0], _ptr(hull_idx, "hull_idx"),
                          _ptr(hull_count, "hull_count"), _ptr(ws, "ws"), ws.numel(), _stream(stream)),
           "ch_hull")


def ch_filter_kgon(pts, dirs, ext_out, surv_idx, surv_pts, surv_count, ws, stream=None):
    """K-direction filter polygon; dirs is a (K, 2) float32 CUDA tensor."""
    _check(load().ch_filter_kgon(_ptr(pts, "pts"), pts.shape[0], _ptr(dirs, "dirs"), dirs.shape[0],
                                 _ptr(ext_out, "ext_out"), _ptr(surv_idx, "surv_idx"), _ptr(surv_pts, "surv_pts"),
                                 _ptr(surv_count, "surv_count"), _ptr(ws, "ws"), ws.numel(), _stream(stream)),
           "ch_filter_kgon")


def ch_hull_kgon(pts, dirs, hull_idx, hull_count, ws, stream=None):
    _check(load().ch_hull_kgon(_ptr(pts, "pts"), pts.shape[0], _ptr(dirs, "dirs"), dirs.shape[0],
                               _ptr(hull_idx, "hull_idx"), _ptr(hull_count, "hull_count"), _ptr(ws, "ws"),
                               ws.numel(), _stream(stream)), "ch_hull_kgon")


def ch_hull_octagon_kgon(pts, dirs, K, ext_out, hull_idx, hull_count, ws, stream=None):
    _check(load().ch_hull_octagon_kgon(_ptr(pts, "pts"), pts.shape[0], _ptr(dirs, "dirs"), int(K), _ptr(ext_out, "ext_out"),
                                       _ptr(hull_idx, "hull_idx"), _ptr(hull_count, "hull_count"), _ptr(ws, "ws"),
                                       ws.numel(), _stream(stream)), "ch_hull_octagon_kgon")


def ch_hull_learned(pts, params, dirs_out, k_out, hull_idx, hull_count, ws, stream=None):
    _check(load().ch_hull_learned(_ptr(pts, "pts"), pts.shape[0], _ptr(params, "params"), _ptr(dirs_out, "dirs_out"),
                                  _ptr(k_out, "k_out"), _ptr(hull_idx, "hull_idx"), _ptr(hull_count, "hull_count"),
                                  _ptr(ws, "ws"), ws.numel(), _stream(stream)), "ch_hull_learned")


def ch_hull_batched(pts, offsets, hull_idx, hull_offsets, ws, stream=None):
    _check(load().ch_hull_batched(_ptr(pts, "pts"), _ptr(offsets, "offsets"), offsets.shape[0] - 1,
                                  _ptr(hull_idx, "hull_idx"), _ptr(hull_offsets, "hull_offsets"),
                                  _ptr(ws, "ws"), ws.numel(), _stream(stream)), "ch_hull_batched")


def ch_tune_set(knob: str, value: int):
    """A tuning knob (convhull.h's ch_tune_knob, by name): a batched
    kernel's blocks per SM or launch shape, or the second fan level's
    threshold; 0 restores the built-in choice."""
    _check(load().ch_tune_set(TUNE_KNOBS.index(knob), int(value)), "ch_tune_set")


def ch_tune_get(knob: str) -> int:
    v = ctypes.c_int32()
    _check(load().ch_tune_get(TUNE_KNOBS.index(knob), ctypes.byref(v)), "ch_tune_get")
    return int(v.value)


def ch_hull_counts(ws, n, stream=None):
    """(octagon survivors, points sorted, speculative sweep used: 0/1, points
    left by the fan's first level) of the last ch_hull call for n points on
    ws (instrumentation; synchronises the stream)."""
    out = (ctypes.c_uint32 * 4)()
    _check(load().ch_hull_counts(_ptr(ws, "ws"), ws.numel(), int(n), ctypes.addressof(out), _stream(stream)),
           "ch_hull_counts")
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def ch_last_error(ws, stream=None) -> int:
    """Synchronises the stream; returns (and clears) the device-side status."""
    return int(load().ch_last_error(_ptr(ws, "ws"), _stream(stream)))


def ch_filter_variant(variant: int):
    """Compaction schedule of the filter: 0 two passes (default), 1 single
    pass with decoupled look-back.  Results are identical."""
    _check(load().ch_filter_variant(int(variant)), "ch_filter_variant")


def ch_probe_start(kernels=KERNELS, max_launches: int = 1024):
    """Time every launch of the named kernels with CUDA events (instrumentation)."""
    mask = 0
    for k in kernels:
        mask |= 1 << KERNELS.index(k)
    _check(load().ch_probe_start(mask, int(max_launches)), "ch_probe_start")


def ch_probe_stop():
    """Returns {kernel: (event-timed ms summed over launches, launches)}."""
    ms = (ctypes.c_double * len(KERNELS))()
    ln = (ctypes.c_int64 * len(KERNELS))()
    _check(load().ch_probe_stop(ctypes.addressof(ms), ctypes.addressof(ln)), "ch_probe_stop")
    return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(KERNELS)}


# ---------------------------------------------------------------- conveniences

class Workspace:
    """Zeroed device scratch for problems of up to ``n`` points."""

    def __init__(self, n: int, num_sets: int = 1, device="cuda"):
        import torch
        self.n = int(n)
        self.num_sets = int(num_sets)
        self.nbytes = ch_workspace_size(self.n, self.num_sets)
        self.buf = torch.zeros(self.nbytes, dtype=torch.uint8, device=device)

    def fits(self, n: int, num_sets: int = 1) -> bool:
        return ch_workspace_size(n, num_sets) <= self.nbytes

    def check(self, stream=None):
        rc = ch_last_error(self.buf, stream)
        if rc != CH_OK:
            raise CHError(rc, "device")


def _as_points(pts):
    import torch
    if pts.dtype != torch.float32 or pts.dim() != 2 or pts.shape[1] != 2:
        raise ValueError("points must be an (n, 2) float32 tensor")
    return pts.contiguous()


def extremes(pts, ws: Workspace | None = None):
    """Indices (int32 tensor of 8) of R, TR, T, TL, L, BL, B, BR (Sec. 3.1)."""
    import torch
    pts = _as_points(pts)
    ws = ws or Workspace(pts.shape[0], device=pts.device)
    ext8 = torch.empty(8, dtype=torch.int32, device=pts.device)
    ch_extremes(pts, ext8, ws.buf)
    return ext8


def filter_points(pts, ext8, ws: Workspace | None = None, with_points: bool = True):
    """(surv_idx, surv_pts or None, count) on the device (Sec. 3.2); entries
    beyond ``count`` are unspecified."""
    import torch
    pts = _as_points(pts)
    n = pts.shape[0]
    ws = ws or Workspace(n, device=pts.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    sp = torch.empty((max(n, 1), 2), dtype=torch.float32, device=pts.device) if with_points else None
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
    ch_filter(pts, ext8, idx, sp, cnt, ws.buf)
    return idx, sp, cnt


def extremes_and_filter(pts, ws: Workspace | None = None, with_points: bool = True):
    """(ext8, surv_idx, surv_pts or None, count) on the device from one
    ch_extremes_filter call; entries beyond ``count`` are unspecified."""
    import torch
    pts = _as_points(pts)
    n = pts.shape[0]
    ws = ws or Workspace(n, device=pts.device)
    ext8 = torch.zeros(8, dtype=torch.int32, device=pts.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    sp = torch.empty((max(n, 1), 2), dtype=torch.float32, device=pts.device) if with_points else None
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
    ch_extremes_filter(pts, ext8, idx, sp, cnt, ws.buf)
    return ext8, idx, sp, cnt


def convex_hull(pts, ws: Workspace | None = None):
    """(hull_idx, count) on the device: counter-clockwise hull vertex indices."""
    import torch
    pts = _as_points(pts)
    n = pts.shape[0]
    ws = ws or Workspace(n, device=pts.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
    ch_hull(pts, idx, cnt, ws.buf)
    return idx, cnt


def _as_dirs(dirs, device):
    import torch
    d = torch.as_tensor(dirs, dtype=torch.float32).reshape(-1, 2)
    return d.to(device).contiguous()


def filter_points_kgon(pts, dirs, ws: Workspace | None = None):
    """(vertex indices, surv_idx, surv_pts, count) on the device for the
    K-direction polygon of the (K, 2) directions ``dirs``."""
    import torch
    pts = _as_points(pts)
    n = pts.shape[0]
    d = _as_dirs(dirs, pts.device)
    ws = ws or Workspace(n, device=pts.device)
    ext = torch.zeros(d.shape[0], dtype=torch.int32, device=pts.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    sp = torch.empty((max(n, 1), 2), dtype=torch.float32, device=pts.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
    ch_filter_kgon(pts, d, ext, idx, sp, cnt, ws.buf)
    return ext, idx, sp, cnt


def convex_hull_kgon(pts, dirs, ws: Workspace | None = None):
    """(hull_idx, count) on the device, with the K-direction filter polygon."""
    import torch
    pts = _as_points(pts)
    n = pts.shape[0]
    d = _as_dirs(dirs, pts.device)
    ws = ws or Workspace(n, device=pts.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
    ch_hull_kgon(pts, d, idx, cnt, ws.buf)
    return idx, cnt


def convex_hull_batched(pts, offsets, ws: Workspace | None = None):
    """(hull_idx, hull_offsets) on the device for the sets
    pts[offsets[b]:offsets[b+1]]; set b's hull (set-local indices) is
    hull_idx[hull_offsets[b]:hull_offsets[b+1]]."""
    import torch
    pts = _as_points(pts)
    n = pts.shape[0]
    if offsets.dtype != torch.int64 or offsets.dim() != 1 or offsets.shape[0] < 1:
        raise ValueError("offsets must be a 1-d int64 tensor of num_sets + 1 entries")
    offsets = offsets.to(pts.device).contiguous()
    num_sets = offsets.shape[0] - 1
    ws = ws or Workspace(n, num_sets=max(num_sets, 1), device=pts.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    hoff = torch.zeros(num_sets + 1, dtype=torch.int64, device=pts.device)
    ch_hull_batched(pts, offsets, idx, hoff, ws.buf)
    return idx, hoff
