"""The bench's roofline bookkeeping on CPU: algorithmic bytes per kernel
follow their definitions, the fan group's ALU roofline uses the recorded
instructions per survivor only while kgon.cu is unchanged, and counts only
the sets whose fan ran."""
import copy
import json

import pytest
import torch

import bench

N = 10**8
S = [69, 99_999_997, 94_825_784]     # octagon survivors
T = [69, 16_543_492, 118_191]        # points sorted after the fan


def test_algorithmic_bytes_definitions():
    assert bench.algorithmic_bytes("extremes", N, S, T) == 3 * 8 * N
    assert bench.algorithmic_bytes("filter", N, S, T) == sum(8 * N + 12 * t for t in T)
    # the fan reads the coordinates of the octagon survivors of the sets it ran on
    assert bench.algorithmic_bytes("kgon", N, S, T) == 8 * (S[1] + S[2])
    # the normal set's 69 points are sorted and chained by one block: no sort or chain traffic
    assert bench.algorithmic_bytes("sort_pass", N, S, T) == sum(4 * 24 * t for t in T[1:])
    assert bench.algorithmic_bytes("chain", N, S, T) == sum(12 * t for t in T[1:])
    assert bench.algorithmic_bytes("sort_hist", N, S, T) == sum(4 * t for t in T[1:])
    assert bench.algorithmic_bytes("emit", N, S, T) is None


def test_algorithmic_bytes_with_the_second_fan_level():
    # the circle set's first level left F[1] points, its second level T[1]:
    # the filter wrote F, the fan group read the octagon survivors, then the
    # first level's survivors twice, and copied the second level's
    F = [69, 16_543_492, 118_191]
    T2 = [69, 600_000, 118_191]
    assert bench.algorithmic_bytes("filter", N, S, T2, F) == sum(8 * N + 12 * f for f in F)
    assert bench.algorithmic_bytes("kgon", N, S, T2, F) == (8 * S[1] + 24 * F[1] + 24 * T2[1]) + 8 * S[2]
    assert bench.algorithmic_bytes("sort_pass", N, S, T2, F) == sum(4 * 24 * t for t in T2[1:])


def test_filter_bytes_of_a_set_the_speculative_sweep_served():
    # the normal set's points were read by the extremes sweep: its filter
    # only writes the survivors
    F = [69, 16_543_492, 118_191]
    assert bench.algorithmic_bytes("filter", N, S, T, F, [1, 0, 0]) == 12 * 69 + sum(8 * N + 12 * f for f in F[1:])


def test_traffic_per_launch_takes_each_distributions_ratio():
    rec = {"dram_per_algorithmic_byte": 1.0,
           "per_dist": {"circle": {"dram_per_algorithmic_byte": 1.2}, "displaced": {"dram_per_algorithmic_byte": 1.1}}}
    F = [69, 16_543_492, 118_191]
    got = bench.traffic_per_launch("filter", rec, N, S, T, F, [1, 0, 0], ["normal", "circle", "displaced"], 5, 10)
    want = (1.0 * 12 * 69 + 1.2 * (8 * N + 12 * F[1]) + 1.1 * (8 * N + 12 * F[2])) * 5 / 10
    assert got == int(want)


@pytest.fixture
def one_device(monkeypatch):
    class Props:
        multi_processor_count = 152
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: Props())


FAN_RECORD = {"source": "kgon.cu", "capture": "test record", "dram_per_algorithmic_byte": 1.25,
              "warp_inst_per_survivor": 4.5}


def test_alu_roofline_counts_fan_sets_only(one_device, monkeypatch):
    monkeypatch.setattr(bench, "load_traffic", lambda kernel: FAN_RECORD if kernel == "kgon" else None)
    rec = FAN_RECORD
    steps, launches, ms = 5, 60, 6.0
    r = bench.alu_roofline(ms, launches, steps, N, S, T, {"sm_max_mhz": 2070.0}, None)
    inst = rec["warp_inst_per_survivor"] * (S[1] + S[2]) * steps
    assert r["bound"] == "alu" and r["kernel"] == "kgon"
    assert r["peak"] == pytest.approx(152 * 4 * 2070e6 / 1e12, abs=1e-3)
    assert r["achieved"] == pytest.approx(inst / (ms * 1e-3) / 1e12, abs=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], abs=1e-3)
    assert r["warp_instr_per_launch"] == int(inst / launches)
    # the same launches against the HBM roofline: 8 B per octagon survivor tested
    hbm_peak, _ = bench.peaks()
    gbs = 8 * (S[1] + S[2]) * steps / launches / (ms / launches * 1e-3) / 1e9
    assert r["hbm_achieved_gbs"] == pytest.approx(gbs, abs=0.1)
    assert r["hbm_frac"] == pytest.approx(gbs / hbm_peak, abs=1e-3)


def test_alu_roofline_takes_each_distributions_capture(one_device, monkeypatch):
    rec = dict(FAN_RECORD, per_dist={"circle": {"warp_inst_per_survivor": 5.0, "dram_per_algorithmic_byte": 1.3},
                                     "displaced": {"warp_inst_per_survivor": 3.0, "dram_per_algorithmic_byte": 1.4}})
    monkeypatch.setattr(bench, "load_traffic", lambda kernel: rec if kernel == "kgon" else None)
    steps, launches, ms = 5, 60, 6.0
    r = bench.alu_roofline(ms, launches, steps, N, S, T, {"sm_max_mhz": 2070.0}, None,
                           ["normal", "circle", "displaced"])
    inst = (5.0 * S[1] + 3.0 * S[2]) * steps
    assert r["warp_instr_per_launch"] == int(inst / launches)
    assert r["traffic"] == int((1.3 * 8 * S[1] + 1.4 * 8 * S[2]) * steps / launches)
    # a distribution without its own capture takes the default
    r2 = bench.alu_roofline(ms, launches, steps, N, S, T, {"sm_max_mhz": 2070.0}, None,
                            ["normal", "circle", "gaussians"])
    assert r2["warp_instr_per_launch"] == int((5.0 * S[1] + 4.5 * S[2]) * steps / launches)


def test_alu_roofline_void_when_source_changed(one_device, monkeypatch):
    rec = copy.deepcopy(json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json"))))
    rec["kgon"]["source_sha"] = "0" * 16
    real_load = json.load
    monkeypatch.setattr(bench.json, "load", lambda f: rec if f.name.endswith("traffic.json") else real_load(f))
    assert bench.load_traffic("kgon") is None
    assert bench.alu_roofline(6.0, 60, 5, N, S, T, {"sm_max_mhz": 2070.0}, None) is None
