"""Launch-tuning knobs on the host (no GPU): range checks, defaults, and
the autotuner's JSON cache."""
import ctypes

import pytest

import paper_2303_10581_gb300 as ch
from paper_2303_10581_gb300 import autotune


def test_knobs_round_trip_and_reject_bad_values():
    lib = ch.load()
    try:
        for k in ch.TUNE_KNOBS:
            assert ch.ch_tune_get(k) == 0
            v = {"bx_fan_chunk": 16, "bx_ext_items": 8, "fan2_min_log2": 12}.get(k, 5)
            ch.ch_tune_set(k, v)
            assert ch.ch_tune_get(k) == v
        assert lib.ch_tune_set(len(ch.TUNE_KNOBS), 1) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(ch.TUNE_KNOBS.index("bx_fan_chunk"), 12) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(ch.TUNE_KNOBS.index("bx_ext_items"), 5) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(ch.TUNE_KNOBS.index("fan2_min_log2"), 9) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(ch.TUNE_KNOBS.index("fan2_min_log2"), 32) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(-1, 1) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(0, 65) == ch.CH_ERR_ARG
        assert lib.ch_tune_set(0, -1) == ch.CH_ERR_ARG
        assert lib.ch_tune_get(0, None) == ch.CH_ERR_ARG
    finally:
        autotune.apply({})
    assert autotune.current() == {k: 0 for k in ch.TUNE_KNOBS}


def test_cache_file(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cached("x", path) is None
    autotune.save({"config": {"bx_filter": 4}, "ms_default": 2.0, "ms_best": 1.5}, "x", path)
    autotune.save({"config": {}, "ms_default": 1.0, "ms_best": 1.0}, "y", path)
    assert autotune.load_cached("x", path)["config"] == {"bx_filter": 4}
    assert autotune.load_cached("y", path)["ms_best"] == 1.0
