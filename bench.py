"""Benchmark of the octagon-filter convex hull on GB300.

Workload (one step): the device hull (extremes -> filter -> sort -> chain)
of three synthetic sets of n = 10^8 binary32 points -- Normal(0,1),
unit circle, displaced circle (radius 1 - |Normal(0, 0.01)|) -- i.e. the
single-set workload at 10^8 points for the three study cases of the paper
(Sec. 5).  Inputs (2.4 GB) are larger than L2 and resident in HBM before
the timed region.

Printed: one JSON line (rank 0).  ``value`` is points through the whole
path per second, over all ranks.  ``e2e`` repeats the measurement through
the public API with the inputs copied from pinned host memory and the hull
copied back inside the timed region.  ``roofline`` is for the kernel with
the largest share of device time (event-timed launches inside the timed
region).  ``cpu_baseline`` times the CPU oracle on a bounded sample.

``--impl reference`` times the CPU oracle as the reference arm on host
cores, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpoints/s filtered (HBM GB/s vs peak); end-to-end hull ms, learned vs octagon"
WORKLOAD = "hull of 3 single sets, n=1e8 fp32 each: normal(0,1), unit circle, displaced circle (r=1-|N(0,0.01)|)"
N_POINTS = 100_000_000
ALL_DISTS = ("normal", "circle", "displaced")
DISTS = ALL_DISTS
KERNEL_IDS = ("extremes", "octagon", "filter", "sort_hist", "sort_pass", "chain", "emit", "finish", "kgon")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--copy-streams", type=int, default=2, help="host-to-device copy streams of the e2e step")
    ap.add_argument("--dists", default=",".join(ALL_DISTS),
                    help="subset of the workload's distributions (profiling runs)")
    ap.add_argument("--filter-variant", type=int, default=0, choices=[0, 1],
                    help="compaction schedule: 0 two passes, 1 single pass with look-back")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "prior-art", "kgon", "learned"],
                    help="single: the three 1e8 sets; batched: 4096 uneven sets, batched call vs per-set calls; "
                         "prior-art: extremes + filter against the paper's Thrust/CUB variants (context); "
                         "kgon: K-direction filter polygons against the octagon")
    ap.add_argument("--sets", type=int, default=4096, help="sets of the batched workload")
    ap.add_argument("--train-sets", type=int, default=32, help="training sets per family (learned workload)")
    ap.add_argument("--sequential-sets", action="store_true",
                    help="run the step's sets one after another on one stream (default: one stream and workspace "
                         "per set, the independent hulls overlapping)")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the records of the 10^9-point filter, the batch and the learned proposal")
    ap.add_argument("--autotune", action="store_true",
                    help="batched workload: tune the batched call's launch grids first (cached in JSON)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- ranks

def max_over_ranks(x, device):
    """The maximum of x over all ranks of the default process group (x
    itself when there is none)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, points_per_rank_step, ms_max):
    """Whole-job Gpoints/s: every rank processes its own replica of the
    workload, the job takes as long as its slowest rank."""
    return world * points_per_rank_step / (ms_max * 1e-3) / 1e9


# --------------------------------------------------------------------------- inputs

def make_inputs(n, seed):
    import pointgen
    return [pointgen.make_points(d, n, seed=seed + ALL_DISTS.index(d)) for d in DISTS]


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"clocks_gpu{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            try:
                os.remove(self.path)
            except OSError:
                pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- roofline bookkeeping

SMALL_HULL = 512   # at most this many points to sort: one block sorts and chains them (no sort passes)


def algorithmic_bytes(kernel, n, s_list, t_list, f_list=None, spec_list=None):
    """Bytes a kernel must move in one step (all its launches for the step's
    sets), from the data it reads and writes by definition; s_list holds the
    octagon-filter survivors of each set, t_list the points the hull step
    sorts (the survivors of the fan test as well, when it ran), f_list the
    points left by the fan's first level (t_list when absent: no second
    level), spec_list 1 for the sets the speculative sweep served (their
    points were read by the extremes sweep: the filter only writes its
    survivors; the candidates it re-reads are not counted).  Sets with at
    most SMALL_HULL points to sort run no sort and chain kernels."""
    f_list = t_list if f_list is None else f_list
    spec_list = [0] * len(s_list) if spec_list is None else spec_list
    if kernel == "extremes":
        return sum(8 * n for _ in s_list)                   # read the points
    if kernel == "filter":
        # read points (unless the sweep served), write key + payload per point kept
        return sum((0 if sp else 8 * n) + 12 * f for f, sp in zip(f_list, spec_list))
    if kernel == "kgon":
        # the fan test of the octagon survivors when it ran (read their
        # coordinates); otherwise only samples.  The second level reads the
        # first level's survivors twice (sub-bin maxima, test: key +
        # payload) and copies the points it keeps
        return sum((8 * s if f < s else 0) + (24 * f + 24 * t if t < f else 0)
                   for s, t, f in zip(s_list, t_list, f_list))
    big = [t for t in t_list if t > SMALL_HULL]
    if kernel == "sort_hist":
        return sum(4 * t for t in big)                      # read the 32-bit keys
    if kernel == "sort_pass":
        # 4 passes (32-bit x key) per set; each reads and writes key (4 B)
        # + payload (8 B): 24 B per point
        return sum(4 * 24 * t for t in big)
    if kernel == "chain":
        return sum(12 * t for t in big)                     # read the sorted keys and payloads once
    return None


def load_traffic(kernel):
    """ncu DRAM bytes of a captured launch of `kernel`, as a ratio to that
    launch's algorithmic bytes, recorded under profiles/ -- None when the
    kernel's source file changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel)
        if not rec:
            return None
        src = os.path.join(ROOT, "paper_2303_10581_gb300", "csrc", rec["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if h != rec.get("source_sha"):
            return None
        return rec
    except Exception:
        return None


def fan_rates(tr, dist):
    """(warp instructions, DRAM bytes per algorithmic byte) per octagon
    survivor of the fan kernels for a set of distribution `dist`: the
    capture of that distribution when the record has one, else its
    default."""
    rec = (tr.get("per_dist") or {}).get(dist) or tr
    return rec["warp_inst_per_survivor"], rec["dram_per_algorithmic_byte"]


def traffic_per_launch(kernel, tr, n, s_list, t_list, f_list, spec_list, dists, steps, launches):
    """DRAM bytes per launch of `kernel` from a traffic record: each set's
    algorithmic bytes times the ratio captured for its distribution (the
    record's default for the others)."""
    total = 0.0
    for k in range(len(s_list)):
        one = lambda lst: [lst[k]] if lst is not None else None
        b = algorithmic_bytes(kernel, n, [s_list[k]], [t_list[k]], one(f_list), one(spec_list))
        rec = (tr.get("per_dist") or {}).get(dists[k]) or tr
        total += rec["dram_per_algorithmic_byte"] * b
    return int(total * steps / launches)


def alu_roofline(dom_ms, dom_launches, steps, n, s_list, t_list, clk, dev, dists=None, f_list=None):
    """Roofline of the fan kernels, which are bound by instruction issue,
    not by HBM: warp instructions issued per second against the SMs' issue
    rate (4 warp schedulers per SM, one warp instruction each per clock, at
    the highest SM clock seen).  The instructions per octagon survivor come
    from ncu captures (profiles/traffic.json, per distribution of the
    set, void once kgon.cu changed); the time is the event time of the
    timed launches."""
    import torch

    tr = load_traffic("kgon")
    if not tr or "warp_inst_per_survivor" not in tr:
        return None
    dists = dists or [None] * len(s_list)
    f_list = t_list if f_list is None else f_list
    fan = [(s, d) for s, f, d in zip(s_list, f_list, dists) if f < s]   # sets whose fan pass ran
    inst = sum(fan_rates(tr, d)[0] * s for s, d in fan) * steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    peak = sms * 4 * mhz * 1e6 / 1e12                          # T warp-instructions/s
    achieved = inst / (dom_ms * 1e-3) / 1e12
    per_launch_bytes = algorithmic_bytes("kgon", n, s_list, t_list, f_list) * steps / dom_launches
    hbm_peak, hbm_kind = peaks()
    hbm_gbs = per_launch_bytes / (dom_ms / dom_launches * 1e-3) / 1e9
    return {"kernel": "kgon", "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "T warp-instr/s", "frac": round(achieved / peak, 4),
            "peak_source": f"derived: {sms} SMs x 4 issue slots x {mhz:.0f} MHz",
            # the same launches against the HBM roofline: algorithmic bytes
            # (8 B per octagon survivor tested) over the event time
            "hbm_achieved_gbs": round(hbm_gbs, 1), "hbm_peak_gbs": hbm_peak,
            "hbm_frac": round(hbm_gbs / hbm_peak, 4), "hbm_peak_source": hbm_kind,
            "traffic": int(sum(fan_rates(tr, d)[1] * 8 * s for s, d in fan) * steps / dom_launches),
            "traffic_source": tr["capture"], "algorithmic_bytes_per_launch": int(per_launch_bytes),
            "warp_instr_per_launch": int(inst / dom_launches), "avg_launch_ms": round(dom_ms / dom_launches, 4)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- CPU oracle timing

def cpu_oracle_rate(sample_n, seed):
    import oracle
    pts = make_inputs(sample_n, seed + 100)
    t0 = time.perf_counter()
    for p in pts:
        oracle.convex_hull(p)
    dt = time.perf_counter() - t0
    return len(pts) * sample_n / dt / 1e9, dt


# --------------------------------------------------------------------------- arms

def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    sample_n = 4_000_000
    for _ in range(args.warmup):
        cpu_oracle_rate(sample_n // 10, args.seed)
    times = []
    for _ in range(args.steps):
        rate, dt = cpu_oracle_rate(sample_n, args.seed)
        times.append(dt)
    pts_per_step = 3 * sample_n
    value = pts_per_step * len(times) / sum(times) / 1e9
    sample = f"{sample_n} points of each of the 3 distributions per step (full workload: {args.n} each)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+exact",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "Gpoints/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2303_10581_gb300 as ch

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    host = make_inputs(n, args.seed)
    d_pts = [torch.from_numpy(p).to(dev) for p in host]
    # one workspace per set: the step's hulls are independent problems and
    # run on streams of their own (unless --sequential-sets), so that one
    # set's latency-bound stages overlap another's streaming ones
    wss = ([ch.Workspace(n, device=dev)] * len(DISTS) if args.sequential_sets
           else [ch.Workspace(n, device=dev) for _ in DISTS])
    ch.ch_filter_variant(args.filter_variant)
    hull_idx = [torch.empty(n, dtype=torch.int32, device=dev) for _ in DISTS]
    hull_cnt = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in DISTS]
    stream = torch.cuda.current_stream()
    set_streams = ([stream] * len(DISTS) if args.sequential_sets
                   else [torch.cuda.Stream(device=dev) for _ in DISTS])

    def sequential_step():
        for k in range(len(DISTS)):
            ch.ch_hull(d_pts[k], hull_idx[k], hull_cnt[k], wss[k].buf, stream)

    def step():
        if args.sequential_sets:
            sequential_step()
            return
        start = torch.cuda.Event()
        start.record(stream)
        done = []
        for k in range(len(DISTS)):
            set_streams[k].wait_event(start)
            ch.ch_hull(d_pts[k], hull_idx[k], hull_cnt[k], wss[k].buf, set_streams[k])
            ev = torch.cuda.Event()
            ev.record(set_streams[k])
            done.append(ev)
        for ev in done:
            stream.wait_event(ev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up, then one probed step for the kernel shares and survivor counts
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for w in wss:
        w.check()
    # one probed step, set by set on one stream: event time of every kernel
    per_set = {}
    probe_all = {k: (0.0, 0) for k in KERNEL_IDS}
    surv, sorted_pts, spec, fan1 = [], [], [], []
    for k in range(len(DISTS)):
        ch.ch_probe_start(KERNEL_IDS, max_launches=64)
        ch.ch_hull(d_pts[k], hull_idx[k], hull_cnt[k], wss[k].buf, stream)
        pr = ch.ch_probe_stop()
        per_set[DISTS[k]] = {kk: round(v[0], 4) for kk, v in pr.items() if v[1]}
        probe_all = {kk: (probe_all[kk][0] + pr[kk][0], probe_all[kk][1] + pr[kk][1]) for kk in KERNEL_IDS}
        c = ch.ch_hull_counts(wss[k].buf, n, stream)
        surv.append(c[0])
        sorted_pts.append(c[1])
        spec.append(c[2])
        fan1.append(c[3])
    for w in wss:
        w.check()
    dominant = max(probe_all, key=lambda k: probe_all[k][0])
    total_probe = sum(v[0] for v in probe_all.values())
    shares = {k: round(v[0] / total_probe, 4) for k, v in probe_all.items() if v[1]}
    hull_sizes = [int(c.item()) for c in hull_cnt]

    # timed region: the dominant kernel's launches are event-timed on the
    # streams they are launched on (with the sets overlapping, these times
    # include the other sets' share of the GPU)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    ch.ch_probe_start([dominant], max_launches=64 * args.steps)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    barrier()
    probe = ch.ch_probe_stop()
    clk = clocks.stop()
    for w in wss:
        w.check()
    ms = t0.elapsed_time(t1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    pts_per_step = len(DISTS) * n
    value = job_rate(world, pts_per_step, ms_max)
    launches_per_step = sum(v[1] for v in probe.values()) / args.steps

    # roofline of the dominant kernel: its launch times from a second timed
    # region of K steps with the sets one after another (with the sets
    # overlapping, a launch's event time includes the other sets' share of
    # the GPU); the same K steps, the same events on the launching stream
    if not args.sequential_sets:
        barrier()
        ch.ch_probe_start([dominant], max_launches=64 * args.steps)
        for _ in range(args.steps):
            sequential_step()
        barrier()
        probe = ch.ch_probe_stop()
        for w in wss:
            w.check()
    dom_ms, dom_launches = probe[dominant]
    peak, peak_kind = peaks()
    roof = None
    if dom_launches and dominant == "kgon":
        roof = alu_roofline(dom_ms, dom_launches, args.steps, n, surv, sorted_pts, clk, dev, list(DISTS), fan1)
    if dom_launches and roof is None:
        per_step_bytes = algorithmic_bytes(dominant, n, surv, sorted_pts, fan1, spec)
        if per_step_bytes is not None:
            # algorithmic bytes of all timed launches over their summed event
            # time (= per-launch bytes over the average launch duration)
            per_launch_bytes = per_step_bytes * args.steps / dom_launches
            avg_ms = dom_ms / dom_launches
            achieved = per_step_bytes * args.steps / (dom_ms * 1e-3) / 1e9
            tr = load_traffic(dominant)
            roof = {"kernel": dominant, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                    "traffic": traffic_per_launch(dominant, tr, n, surv, sorted_pts, fan1, spec, list(DISTS),
                                                  args.steps, dom_launches) if tr else None,
                    "traffic_source": tr["capture"] if tr else None,
                    "algorithmic_bytes_per_launch": int(per_launch_bytes), "avg_launch_ms": round(avg_ms, 4)}

    # filter-only throughput (the paper's headline stage) from its own launches
    filt = None
    if probe_all["filter"][1]:
        fms = probe_all["filter"][0]
        fb = algorithmic_bytes("filter", n, surv, sorted_pts, fan1, spec)
        filt = {"gpoints_s": round(pts_per_step / (fms * 1e-3) / 1e9, 2), "ms_per_set": round(fms / len(DISTS), 4),
                "gbs": round(fb / (fms * 1e-3) / 1e9, 1), "frac_of_peak": round(fb / (fms * 1e-3) / 1e9 / peak, 4)}

    # end to end through the public API: pinned host -> device, hull, device -> host
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(p).pin_memory() for p in host]
        out_host = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in DISTS]
        cnt_host = [torch.empty(1, dtype=torch.int32).pin_memory() for _ in DISTS]

        # copies and hulls overlap: every set's points go up in equal parts
        # on several copy streams while the compute stream works on the
        # previous set; the set with the shortest hull goes last
        nc = max(1, args.copy_streams)
        copy_streams = [torch.cuda.Stream(device=dev) for _ in range(nc)]
        order = sorted(range(len(DISTS)), key=lambda k: -sum(per_set[DISTS[k]].values()))
        cuts = [n * c // nc for c in range(nc + 1)]

        def e2e_step():
            d2h = 0
            ready = []
            for k in order:
                evs = []
                for c in range(nc):
                    lo, hi = cuts[c], cuts[c + 1]
                    with torch.cuda.stream(copy_streams[c]):
                        d_pts[k][lo:hi].copy_(pinned[k][lo:hi], non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(copy_streams[c])
                        evs.append(ev)
                ready.append(evs)
            for k, evs in zip(order, ready):
                for ev in evs:
                    stream.wait_event(ev)
                ch.ch_hull(d_pts[k], hull_idx[k], hull_cnt[k], wss[k].buf, stream)
                cnt_host[k].copy_(hull_cnt[k], non_blocking=True)
            stream.synchronize()
            for k in range(len(DISTS)):
                h = int(cnt_host[k].item())
                out_host[k][:h].copy_(hull_idx[k][:h], non_blocking=True)
                d2h += 4 + 4 * h
            stream.synchronize()
            return d2h

        e2e_step()
        barrier()
        w0 = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            d2h = e2e_step()
        barrier()
        e_ms = max_over_ranks((time.perf_counter() - w0) * 1e3 / args.steps, dev)
        e2e = {"value": round(job_rate(world, pts_per_step, e_ms), 3), "unit": "Gpoints/s",
               "ms_per_step": round(e_ms, 3), "h2d_bytes_per_step": 8 * n * len(DISTS),
               "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sample_n = 20_000_000   # about 10 s of single-core oracle work
        rate, dt = cpu_oracle_rate(sample_n, args.seed)
        cpu = {"value": round(rate, 5), "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
               "sample": f"{sample_n} points of each distribution (3 sets), whole path, {dt:.1f} s"}

    # the other configurations of the metric, one record each (one GPU only;
    # outside the timed region above)
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        extra["filter_1e9"] = filter_1e9_record(dev, stream, max(5, args.steps), args.warmup, peak, peak_kind)
        extra["batched"] = batched_record(dev, stream, max(5, args.steps), args.warmup)
        extra["learned_vs_octagon"] = learned_record(dev, stream, n, 3, 2, args.train_sets, args.seed)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gpoints/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+exact", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_per_set": n, "sets_per_step": len(DISTS),
                       "sets_schedule": ("one after another, one stream" if args.sequential_sets
                                         else "one stream and workspace per set, overlapping"),
                       "roofline_timing": ("the timed region" if args.sequential_sets else
                                           "a second timed region of the same steps, sets one after another"),
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (2.4 GB)",
                       "survivors": dict(zip(DISTS, surv)), "sorted": dict(zip(DISTS, sorted_pts)),
                       "speculative_sweep": dict(zip(DISTS, spec)),
                       "fan_first_level": dict(zip(DISTS, fan1)),
                       "hull_sizes": dict(zip(DISTS, hull_sizes))},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roof, "filter": filt, "kernel_shares": shares, "kernel_ms_per_set": per_set,
            "hull_ms_per_set": {d: round(sum(v.values()), 4) for d, v in per_set.items()},
            "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


BATCH_WORKLOAD = ("{B} independent sets, sizes log-uniform in [1e2, 1e6] points, distribution drawn from "
                  "normal / circle / displaced circle, scaled by U[0.1, 10], rotated by U[0, 2 pi)")

# --------------------------------------------------------------------------- the other configurations

N_1E9 = 1_000_000_000


def ev_time(fn, steps, warmup, stream):
    """Average ms of one call of fn: CUDA events on `stream` around `steps`
    calls, after `warmup` untimed calls, synchronised on both sides."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps


def _rate(bytes_, ms, peak):
    gbs = bytes_ / (ms * 1e-3) / 1e9
    return round(gbs, 1), round(gbs / peak, 4)


def filter_1e9_record(dev, stream, steps, warmup, peak, peak_kind):
    """The 10^9-point configuration (8 GB of packed float2, Normal(0,1),
    seed 1 -- the set the large parity test compares with the oracle):
    ch_extremes, then ch_filter with each compaction schedule, then
    ch_hull, each timed alone with CUDA events over `steps` calls (the
    input is larger than L2).  GB/s from algorithmic bytes: 8 B per point
    read, 12 B per survivor written (index + point)."""
    import torch

    import paper_2303_10581_gb300 as ch
    import pointgen

    n = N_1E9
    host = pointgen.make_points_blocked("normal", n, seed=1)
    d = torch.from_numpy(host).to(dev)
    del host
    ws = ch.Workspace(n, device=dev)
    ext = torch.zeros(8, dtype=torch.int32, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    sp = torch.empty((n, 2), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    rec = {"workload": "single set, n=1e9 fp32 Normal(0,1), seed 1 (8 GB packed float2, larger than L2)",
           "peak_gbs": peak, "peak_source": peak_kind, "steps": steps, "warmup": warmup}
    e_ms = ev_time(lambda: ch.ch_extremes(d, ext, ws.buf, stream), steps, warmup, stream)
    gbs, frac = _rate(8 * n, e_ms, peak)
    rec["extremes"] = {"ms": round(e_ms, 4), "gbs": gbs, "frac_of_peak": frac}
    for variant, name in ((0, "two_pass"), (1, "single_pass")):
        ch.ch_filter_variant(variant)
        try:
            f_ms = ev_time(lambda: ch.ch_filter(d, ext, idx, sp, cnt, ws.buf, stream), steps, warmup, stream)
        finally:
            ch.ch_filter_variant(0)
        ws.check()
        s = int(cnt.item())
        gbs, frac = _rate(8 * n + 12 * s, f_ms, peak)
        rec[name] = {"ms": round(f_ms, 4), "gpoints_s": round(n / (f_ms * 1e-3) / 1e9, 1), "gbs": gbs,
                     "frac_of_peak": frac, "survivors": s}
    h_ms = ev_time(lambda: ch.ch_hull(d, idx, cnt, ws.buf, stream), steps, warmup, stream)
    ws.check()
    rec["hull"] = {"ms": round(h_ms, 4), "gpoints_s": round(n / (h_ms * 1e-3) / 1e9, 1),
                   "hull_vertices": int(cnt.item())}
    rec["target_0.7_met"] = rec["two_pass"]["frac_of_peak"] >= 0.7
    del d, ws, idx, sp
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def batched_record(dev, stream, steps, warmup, B=4096, seed=1):
    """The batched configuration: one ch_hull_batched call over B uneven
    sets, captured in a CUDA graph, graph replays timed with CUDA events
    (inputs 3.6 GB, larger than L2).  Launch grids: the autotuner's cached
    choice for this GPU and batch shape when there is one, else the
    built-in ones."""
    import torch

    import paper_2303_10581_gb300 as ch
    import pointgen
    from paper_2303_10581_gb300 import autotune

    pts, offsets, _ = pointgen.make_batch(B, seed=seed)
    n = len(pts)
    d_pts = torch.from_numpy(pts).to(dev)
    d_off = torch.from_numpy(offsets).to(dev)
    del pts
    ws = ch.Workspace(n, num_sets=B, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    hoff = torch.zeros(B + 1, dtype=torch.int64, device=dev)
    saved = autotune.current()
    cached = autotune.load_cached(autotune.cache_key(dev, B, n))
    if cached:
        autotune.apply(cached)
    try:
        ch.ch_hull_batched(d_pts, d_off, idx, hoff, ws.buf, stream)
        torch.cuda.synchronize()
        ws.check()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            ch.ch_hull_batched(d_pts, d_off, idx, hoff, ws.buf)
        ms = ev_time(graph.replay, steps, warmup, stream)
        ws.check()
        ch.ch_probe_start(ch.KERNELS, max_launches=64)
        ch.ch_hull_batched(d_pts, d_off, idx, hoff, ws.buf, stream)
        launches = sum(v[1] for v in ch.ch_probe_stop().values())
        ws.check()
    finally:
        autotune.apply(saved)
    rec = {"workload": BATCH_WORKLOAD.format(B=B) + f", seed {seed}", "points": int(n), "sets": B,
           "graph_replay_ms": round(ms, 4), "gpoints_s": round(n / (ms * 1e-3) / 1e9, 2),
           "hull_vertices": int(hoff[-1].item()), "gpu_launches_per_batch": int(launches),
           "launch_grids": "autotuned (cached)" if cached else "built-in"}
    del graph, d_pts, d_off, ws, idx
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec




def run_batched(args):
    """The batched workload: one ch_hull_batched call (direct, and replayed
    from a CUDA graph) against one ch_hull call per set, end to end on
    resident inputs; the per-set hulls of both must agree exactly."""
    import numpy as np
    import torch

    import paper_2303_10581_gb300 as ch
    import pointgen

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B = args.sets
    pts, offsets, _ = pointgen.make_batch(B, seed=args.seed)
    n = len(pts)
    d_pts = torch.from_numpy(pts).to(dev)
    d_off = torch.from_numpy(offsets).to(dev)
    stream = torch.cuda.current_stream()
    ws = ch.Workspace(n, num_sets=B, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    hoff = torch.zeros(B + 1, dtype=torch.int64, device=dev)
    sizes = np.diff(offsets)
    ws1 = ch.Workspace(int(sizes.max()), device=dev)
    idx1 = torch.empty(n, dtype=torch.int32, device=dev)
    cnt1 = torch.zeros(B, dtype=torch.int32, device=dev)
    views = [(d_pts[offsets[b]:offsets[b + 1]], idx1[offsets[b]:offsets[b + 1]], cnt1[b:b + 1]) for b in range(B)]

    def batched():
        ch.ch_hull_batched(d_pts, d_off, idx, hoff, ws.buf, stream)

    def per_set():
        for v, o, c in views:
            if v.shape[0]:
                ch.ch_hull(v, o, c, ws1.buf, stream)

    def timed(fn, steps):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    for _ in range(args.warmup):
        batched()
        per_set()
    ws.check()
    ws1.check()
    # both forms give the same hull for every set
    h_b = hoff.cpu().numpy()
    ib = idx.cpu().numpy()
    i1 = idx1.cpu().numpy()
    c1 = cnt1.cpu().numpy()
    for b in range(B):
        assert h_b[b + 1] - h_b[b] == c1[b], b
        assert np.array_equal(ib[h_b[b]:h_b[b + 1]], i1[offsets[b]:offsets[b] + c1[b]]), b

    tuned = None
    if args.autotune:
        from paper_2303_10581_gb300 import autotune
        tuned = autotune.tune(d_pts, d_off, ws)          # leaves the best grids applied
        autotune.save(tuned, autotune.cache_key(dev, B, n))
        batched()
        torch.cuda.synchronize()
        ws.check()
        assert np.array_equal(hoff.cpu().numpy(), h_b) and np.array_equal(idx.cpu().numpy()[: h_b[-1]], ib[: h_b[-1]])

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ch.ch_hull_batched(d_pts, d_off, idx, hoff, ws.buf)
    graph.replay()
    torch.cuda.synchronize()
    ws.check()
    assert np.array_equal(hoff.cpu().numpy(), h_b)

    ms_batched = timed(batched, args.steps)
    ms_graph = timed(graph.replay, args.steps)
    ms_loop = timed(per_set, max(1, args.steps // 2))
    ch.ch_probe_start(ch.KERNELS, max_launches=64)
    batched()
    launches = sum(v[1] for v in ch.ch_probe_stop().values())
    ws.check()
    line = {
        "metric": "end-to-end hull time of a batch of uneven sets: batched call vs one call per set",
        "value": round(ms_graph, 4), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "dtype": "f32+exact", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(B=B), "points": int(n), "sets": B,
                   "largest_set": int(sizes.max()), "hull_vertices": int(h_b[-1])},
        "batched_graph_ms": round(ms_graph, 4), "batched_ms": round(ms_batched, 4),
        "per_set_calls_ms": round(ms_loop, 4), "speedup_vs_per_set": round(ms_loop / ms_graph, 2),
        "gpoints_s": round(n / (ms_graph * 1e-3) / 1e9, 3), "gpu_launches_per_batch": int(launches),
        "autotune": tuned,
    }
    print(json.dumps(line), flush=True)


PRIOR_VARIANTS = ("cub-flagged", "thrust-copy", "thrust-scan")


def run_prior_art(args):
    """Context for the paper's library variants (Sec. 4): each set's extremes
    + filter + compaction done with Thrust / CUB calls (cub-flagged,
    thrust-copy, thrust-scan, with the paper's plain binary32 point test;
    libpriorart) against this library's ch_extremes + ch_filter (exact
    test), on the same resident inputs, CUDA events over the calls."""
    import ctypes

    import torch

    import paper_2303_10581_gb300 as ch
    from paper_2303_10581_gb300 import build as build_mod

    lib = ctypes.CDLL(build_mod.build_prior_art())
    lib.pa_workspace_size.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    lib.pa_filter.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n = args.n
    host = make_inputs(n, args.seed)
    size = ctypes.c_size_t()
    assert lib.pa_workspace_size(n, ctypes.byref(size)) == 0
    pws = torch.empty(size.value, dtype=torch.uint8, device=dev)
    ws = ch.Workspace(n, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    out_pts = torch.empty((n, 2), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    ext = torch.zeros(8, dtype=torch.int32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / args.steps

    per_set = {}
    for k, dist in enumerate(DISTS):
        d = torch.from_numpy(host[k]).to(dev)

        def ours():
            ch.ch_extremes(d, ext, ws.buf, stream)
            ch.ch_filter(d, ext, out, out_pts, cnt, ws.buf, stream)

        row = {"this library": {"ms": round(timed(ours), 4), "survivors": int(cnt.item())}}
        ws.check()
        for v, name in enumerate(PRIOR_VARIANTS):
            def lib_variant(v=v):
                rc = lib.pa_filter(d.data_ptr(), n, v, out.data_ptr(), cnt.data_ptr(), pws.data_ptr(), size.value,
                                   stream.cuda_stream)
                assert rc == 0, (name, rc)

            row[name] = {"ms": round(timed(lib_variant), 4), "survivors": int(cnt.item())}
        for r in row.values():
            r["gpoints_s"] = round(n / (r["ms"] * 1e-3) / 1e9, 2)
        per_set[dist] = row
        del d
    ours_ms = sum(per_set[d]["this library"]["ms"] for d in DISTS) / len(DISTS)
    best_lib = {name: sum(per_set[d][name]["ms"] for d in DISTS) / len(DISTS) for name in PRIOR_VARIANTS}
    line = {
        "metric": "extremes + filter + compaction per set: this library vs the paper's Thrust/CUB variants (context)",
        "value": round(ours_ms, 4), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"one set of n={n} per distribution: " + ", ".join(DISTS), "n_per_set": n,
                   "note": "library variants use the paper's plain binary32 test, this library the exact one"},
        "ms_per_set_mean": {"this library": round(ours_ms, 4), **{k: round(v, 4) for k, v in best_lib.items()}},
        "per_set": per_set,
    }
    print(json.dumps(line), flush=True)


KGON_KS = (8, 16, 32, 64)


def run_kgon(args):
    """The K-direction filter polygon against the plain octagon, on the
    same resident sets: the filter stage (extremes + test + compaction of
    indices and points) and the end-to-end hull, ms per set by CUDA events,
    with the survivors of each polygon -- the timings a learned proposal of
    K would be trained on.  Directions: angles 2 pi k / K, no offsets."""
    import torch

    import paper_2303_10581_gb300 as ch
    import pointgen

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n = args.n
    host = make_inputs(n, args.seed)
    ws = ch.Workspace(n, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    out_pts = torch.empty((n, 2), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    ext = torch.zeros(64, dtype=torch.int32, device=dev)
    dirs = {K: torch.from_numpy(pointgen.kgon_directions(K)).to(dev) for K in KGON_KS}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return round(t0.elapsed_time(t1) / args.steps, 4)

    per_set = {}
    for k, dist in enumerate(DISTS):
        d = torch.from_numpy(host[k]).to(dev)
        row = {}

        def oct_filter():
            ch.ch_extremes(d, ext[:8], ws.buf, stream)
            ch.ch_filter(d, ext[:8], out, out_pts, cnt, ws.buf, stream)

        def oct_hull():
            ch.ch_hull(d, out, cnt, ws.buf, stream)

        f_ms = timed(oct_filter)
        s = int(cnt.item())
        h_ms = timed(oct_hull)
        row["octagon"] = {"filter_ms": f_ms, "survivors": s, "hull_ms": h_ms, "hull": int(cnt.item()),
                          "hull_note": "ch_hull: octagon filter, fan test, sort, chain"}
        for K in KGON_KS:
            def kf(K=K):
                ch.ch_filter_kgon(d, dirs[K], ext[:K], out, out_pts, cnt, ws.buf, stream)

            def kh(K=K):
                ch.ch_hull_kgon(d, dirs[K], out, cnt, ws.buf, stream)

            f_ms = timed(kf)
            s = int(cnt.item())
            h_ms = timed(kh)
            row[f"K={K}"] = {"filter_ms": f_ms, "survivors": s, "hull_ms": h_ms, "hull": int(cnt.item())}
        ws.check()
        per_set[dist] = row
        del d
    line = {
        "metric": "K-direction filter polygon vs the octagon: filter-stage and end-to-end hull ms per set",
        "value": round(sum(per_set[d]["octagon"]["hull_ms"] for d in DISTS) / len(DISTS), 4), "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "dtype": "f32+exact", "data": "synthetic",
        "config": {"workload": f"one set of n={n} per distribution: " + ", ".join(DISTS), "n_per_set": n,
                   "directions": "angles 2 pi k / K, axis and diagonal keys as the octagon's",
                   "note": "ch_hull_kgon sorts every survivor of its polygon (no fan test)"},
        "per_set": per_set,
    }
    print(json.dumps(line), flush=True)


def learned_record(dev, stream, n, steps, warmup, train_sets, seed):
    """The learned proposal against the plain octagon, end-to-end hull time
    on the same GPU.  The proposal: the weights trained by
    ``python -m paper_2303_10581_gb300.learned`` (labels from timings of
    every choice through the method itself: the octagon with the hull
    step's fan, or the octagon then a K-gon over its survivors, K = 16, 32,
    64) when that file exists, else a short training here on 2^20-point
    sets.  Evaluation on one n-point set per family: ch_hull_learned
    (features, MLP, choice and hull on the device, no host synchronisation)
    against ch_hull (octagon + fan).  The hulls must be equal."""
    import numpy as np
    import torch

    import paper_2303_10581_gb300 as ch
    import pointgen
    from paper_2303_10581_gb300 import learned

    t0 = time.perf_counter()
    if os.path.exists(learned.DEFAULT_WEIGHTS):
        prop, meta = learned.load_params(learned.DEFAULT_WEIGHTS, device=dev)
        training = dict(meta, source="weights file " + os.path.relpath(learned.DEFAULT_WEIGHTS, ROOT))
    else:
        n_train = 1 << 20
        prop = learned.Proposal(device=dev, seed=seed)
        ws_small = ch.Workspace(n_train, device=dev)
        sets = [pointgen.make_family(kind, n_train, seed=10_000 * k + s)
                for k, kind in enumerate(pointgen.FAMILIES) for s in range(train_sets)]
        X, label, off, mask = learned.make_labels(sets, ws_small, prop, seed=seed)
        del ws_small, sets
        hist = prop.train(X, label, off, mask, steps=400, batch=48, lr=3e-3, lam=0.5)
        training = {"source": f"trained here: {len(pointgen.FAMILIES) * train_sets} sets of n=2^20",
                    "label_counts_K8_16_32_64": np.bincount(label.cpu().numpy(), minlength=4).tolist(),
                    "final_loss": round(float(np.mean(hist[-20:])), 4)}
    setup_s = time.perf_counter() - t0

    ws = ch.Workspace(n, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return round(e0.elapsed_time(e1) / steps, 4)

    per_family = {}
    for k, kind in enumerate(pointgen.FAMILIES):
        d = torch.from_numpy(pointgen.make_family(kind, n, seed=90 + k)).to(dev)
        ms_fan = timed(lambda: ch.ch_hull(d, out, cnt, ws.buf, stream))
        h_fan = out[: int(cnt.item())].clone()
        res = {}

        bufs = prop.outputs(n, dev)   # (allocated outside the timed calls, as ch_hull's)

        def learned_hull():
            res["h"] = prop.hull_on_device(d, ws, stream, sync=False, out=bufs)

        ms_l = timed(learned_hull)
        idx_l, cnt_l, k_l, _ = res["h"]
        ws.check()
        h_l = idx_l[: int(cnt_l.item())]
        assert torch.equal(h_fan, h_l), kind
        per_family[kind] = {"learned_ms": ms_l, "learned_K": int(k_l.item()), "octagon_with_fan_ms": ms_fan,
                            "learned_over_octagon": round(ms_l / ms_fan, 4), "hull_vertices": int(h_fan.numel())}
        del d
    del ws, out
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    mean_l = sum(v["learned_ms"] for v in per_family.values()) / len(per_family)
    return {
        "workload": f"one set of n={n} per family: " + ", ".join(pointgen.FAMILIES),
        "training": training, "setup_seconds": round(setup_s, 1), "learned_ms_mean": round(mean_l, 4),
        "octagon_with_fan_ms_mean": round(sum(v["octagon_with_fan_ms"] for v in per_family.values())
                                          / len(per_family), 4),
        "per_family": per_family,
    }


def run_learned(args):
    """The learned workload alone (one JSON line); see learned_record."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    rec = learned_record(dev, stream, args.n, args.steps, args.warmup, args.train_sets, args.seed)
    line = {
        "metric": "end-to-end hull ms: learned K-gon proposal vs the plain octagon (same GPU)",
        "value": rec["learned_ms_mean"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "dtype": "f32+exact; MLP bf16 weights, f32 accumulate",
        "data": "synthetic",
        "config": {k: rec[k] for k in ("workload", "training", "setup_seconds")},
        "per_family": rec["per_family"],
    }
    print(json.dumps(line), flush=True)


def main():
    global DISTS
    args = parse()
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "prior-art":
        DISTS = tuple(d for d in args.dists.split(",") if d)
        run_prior_art(args)
        return
    if args.workload == "learned":
        run_learned(args)
        return
    if args.workload == "kgon":
        DISTS = tuple(d for d in args.dists.split(",") if d)
        run_kgon(args)
        return
    DISTS = tuple(d for d in args.dists.split(",") if d)
    assert DISTS and all(d in ALL_DISTS for d in DISTS), args.dists
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
