"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point declared in include/*.h; host argument checks
return their documented status without touching the device."""
import ctypes
import glob
import os
import re

import pytest

import paper_2303_10581_gb300 as ch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(?:ch_status|int32_t|int64_t)\s+(ch_\w+)\s*\(", text))
    return names


def test_header_declares_the_entry_points():
    assert declared_symbols() == set(ch.SYMBOLS)


def test_library_exports_every_declared_symbol():
    lib = ch.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_size_is_monotone_and_host_only():
    sizes = [ch.ch_workspace_size(n) for n in (0, 1, 4096, 4097, 10**6, 10**8)]
    assert all(a <= b for a, b in zip(sizes, sizes[1:]))
    assert sizes[-1] > 24 * 10**8   # sort buffers dominate


def test_host_argument_errors():
    lib = ch.load()
    out = ctypes.c_size_t(0)
    assert lib.ch_workspace_size(-1, 1, ctypes.byref(out)) == ch.CH_ERR_ARG
    assert lib.ch_workspace_size(10, 0, ctypes.byref(out)) == ch.CH_ERR_ARG
    assert lib.ch_workspace_size(1 << 33, 1, ctypes.byref(out)) == ch.CH_ERR_CAPACITY
    assert lib.ch_extremes(None, 10, None, None, 0, None) == ch.CH_ERR_ARG
    assert lib.ch_extremes(8, 0, 16, 256, 1 << 20, None) == ch.CH_ERR_ARG          # n < 1
    assert lib.ch_extremes(4, 10, 16, 256, 1 << 20, None) == ch.CH_ERR_ARG         # pts misaligned
    assert lib.ch_extremes(8, 10, 16, 256, 16, None) == ch.CH_ERR_CAPACITY         # ws too small
    assert lib.ch_extremes(8, 10, 16, 100, 1 << 20, None) == ch.CH_ERR_ARG         # ws misaligned
    assert lib.ch_filter(8, 10, 16, 32, None, None, 256, 1 << 20, None) == ch.CH_ERR_ARG   # no count
    assert lib.ch_hull(8, 1 << 30, 16, 32, 256, 1 << 40, None) == ch.CH_ERR_CAPACITY
    assert lib.ch_hull(8, 10, 16, None, 256, 1 << 20, None) == ch.CH_ERR_ARG
    assert lib.ch_last_error(None, None) == ch.CH_ERR_ARG


def test_workspace_size_grows_with_sets():
    one = ch.ch_workspace_size(10**6, 1)
    many = ch.ch_workspace_size(10**6, 4096)
    assert many > one
    # per-set state is bounded: a few hundred bytes plus one ragged tile's
    # chain buffers per set
    assert many - one < 4096 * 200 * 1024


def test_batched_host_argument_errors():
    lib = ch.load()
    big = 1 << 40
    # hull_batched(pts, offsets, num_sets, hull_idx, hull_offsets, ws, ws_bytes, stream)
    assert lib.ch_hull_batched(8, 8, -1, 16, 8, 256, big, None) == ch.CH_ERR_ARG
    assert lib.ch_hull_batched(8, None, 4, 16, 8, 256, big, None) == ch.CH_ERR_ARG
    assert lib.ch_hull_batched(8, 8, 4, 16, None, 256, big, None) == ch.CH_ERR_ARG
    assert lib.ch_hull_batched(8, 12, 4, 16, 8, 256, big, None) == ch.CH_ERR_ARG    # offsets misaligned
    assert lib.ch_hull_batched(None, 8, 4, 16, 8, 256, big, None) == ch.CH_ERR_ARG
    assert lib.ch_hull_batched(8, 8, 4, 16, 8, None, big, None) == ch.CH_ERR_ARG
    assert lib.ch_hull_batched(8, 8, 4, 16, 8, 100, big, None) == ch.CH_ERR_ARG     # ws misaligned
    assert lib.ch_hull_batched(8, 8, 4, 16, 8, 256, 1024, None) == ch.CH_ERR_CAPACITY


def test_kgon_entry_points_reject_bad_arguments_on_the_host():
    lib = ch.load()
    one = ctypes.c_void_p(256)   # never dereferenced: the checks fail first
    for K in (0, 7, 12, 128):
        assert lib.ch_filter_kgon(one, 10, one, K, None, one, None, one, one, 1 << 30, None) == ch.CH_ERR_ARG
        assert lib.ch_hull_kgon(one, 10, one, K, one, one, one, 1 << 30, None) == ch.CH_ERR_ARG
    assert lib.ch_filter_kgon(one, 10, None, 16, None, one, None, one, one, 1 << 30, None) == ch.CH_ERR_ARG
    assert lib.ch_filter_kgon(one, -1, one, 16, None, one, None, one, one, 1 << 30, None) == ch.CH_ERR_ARG
    assert lib.ch_hull_kgon(one, 10, one, 16, one, None, one, 1 << 30, None) == ch.CH_ERR_ARG
