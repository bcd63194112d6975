"""The learned proposal of the K-direction filter polygon.

A small MLP reads the 32 x 32 occupancy grid of a 4096-point sample of a
point set and picks the direction count K in {8, 16, 32, 64} and the angular
offsets of the polygon; the hull is then ``ch_hull_kgon`` with that polygon,
exact whatever the choice (every vertex is an extreme input point).  The
features, the MLP's forward pass, its backward pass and its Adam step run
in the library's kernels (``ch_kgon_features``, ``ch_mlp_forward``,
``ch_mlp_train_step``); this module marshals buffers, builds the
directions (angles in binary64, rounded once) and generates training labels
from timings of the plain K-gon path itself.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import _check, _ptr, _stream, load

KS = (8, 16, 32, 64)
SPREAD = 0.45          # offsets are in units of pi / K, within (-SPREAD, SPREAD)
N_OFF = 64
_OCTAGON = ((1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1))


def directions(K: int, units=None) -> np.ndarray:
    """(K, 2) binary32 directions at angles 2 pi k / K + units_k * pi / K
    (cos and sin in binary64, rounded once); a multiple of pi / 4 with zero
    offset takes the octagon's integer direction, so K = 8 without offsets
    is the octagon."""
    u = np.zeros(K) if units is None else np.asarray(units, np.float64)[:K]
    out = np.empty((K, 2), np.float32)
    for k in range(K):
        if u[k] == 0.0 and (8 * k) % K == 0:
            out[k] = _OCTAGON[8 * k // K]
        else:
            th = 2.0 * math.pi * k / K + float(u[k]) * math.pi / K
            out[k] = (math.cos(th), math.sin(th))
    return out


class Proposal:
    """The MLP's parameters on the device: BF16 weights (what the kernels
    read), FP32 master weights and Adam moments (training)."""

    def __init__(self, device="cuda", seed: int = 0):
        import torch
        lib = load()
        self.device = torch.device(device)
        self.n_params = int(lib.ch_mlp_param_count())
        rng = np.random.Generator(np.random.PCG64(seed))
        parts = []
        for fan_in, fan_out in ((1024, 64), (64, 64), (64, 68)):   # He-uniform weights, zero biases
            a = math.sqrt(6.0 / fan_in)
            parts += [rng.uniform(-a, a, fan_in * fan_out), np.zeros(fan_out)]
        w = np.concatenate(parts).astype(np.float32)
        assert w.size == self.n_params
        self.master = torch.from_numpy(w).to(self.device)
        self.params = self.master.to(torch.bfloat16)   # round to nearest even, as the update kernel does
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.step = 0

    # -- features and inference -------------------------------------------
    def features(self, pts, out=None, stream=None):
        import torch
        out = torch.empty(1024, dtype=torch.float32, device=pts.device) if out is None else out
        _check(load().ch_kgon_features(_ptr(pts, "pts"), pts.shape[0], _ptr(out, "feat"), _stream(stream)),
               "ch_kgon_features")
        return out

    def forward(self, X, stream=None):
        import torch
        X = X.reshape(-1, 1024).contiguous()
        B = X.shape[0]
        h1 = torch.empty((B, 64), dtype=torch.float32, device=X.device)
        h2 = torch.empty((B, 64), dtype=torch.float32, device=X.device)
        out = torch.empty((B, 68), dtype=torch.float32, device=X.device)
        _check(load().ch_mlp_forward(_ptr(X, "X"), B, _ptr(self.params, "params"), _ptr(h1, "H1"),
                                     _ptr(h2, "H2"), _ptr(out, "OUT"), _stream(stream)), "ch_mlp_forward")
        return out

    def propose(self, pts, stream=None):
        """(K, offsets in units of pi / K) for the point set pts."""
        out = self.forward(self.features(pts, stream=stream), stream).cpu().numpy()[0]
        K = KS[int(np.argmax(out[:4]))]
        return K, np.clip(out[4:4 + K], -SPREAD, SPREAD)

    def hull(self, pts, ws, stream=None):
        """(hull_idx, hull_count, K) with the proposed polygon."""
        import torch
        from . import ch_hull_kgon
        K, units = self.propose(pts, stream)
        d = torch.from_numpy(directions(K, units)).to(pts.device)
        idx = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=pts.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
        ch_hull_kgon(pts, d, idx, cnt, ws.buf, stream)
        return idx, cnt, K

    def outputs(self, n, device):
        """Output buffers for hull_on_device: (hull_idx, hull_count, K,
        directions)."""
        import torch
        return (torch.empty(max(n, 1), dtype=torch.int32, device=device),
                torch.zeros(1, dtype=torch.int32, device=device),
                torch.zeros(1, dtype=torch.int32, device=device),
                torch.empty(128, dtype=torch.float32, device=device))

    def hull_on_device(self, pts, ws, stream=None, sync=True, out=None):
        """ch_hull_learned: features, MLP, the choice of K and directions and
        the hull with that second polygon, all on the device (no host
        synchronisation inside the call).  out: buffers from outputs() (else
        new ones).  Returns (hull_idx, hull_count, K, directions (64, 2)) --
        K and directions read back when sync."""
        from . import ch_hull_learned
        idx, cnt, k, dirs = out if out is not None else self.outputs(pts.shape[0], pts.device)
        ch_hull_learned(pts, self.params, dirs, k, idx, cnt, ws.buf, stream)
        if not sync:
            return idx, cnt, k, dirs
        return idx, cnt, int(k.item()), dirs.cpu().numpy().reshape(64, 2)

    # -- training ----------------------------------------------------------
    def train_step(self, X, label, off, mask, lam=1.0, lr=1e-3, scratch=None, loss=None, stream=None):
        import torch
        lib = load()
        B = X.shape[0]
        scratch = scratch if scratch is not None else torch.empty(
            int(lib.ch_mlp_scratch_floats(B)), dtype=torch.float32, device=X.device)
        loss = loss if loss is not None else torch.empty(B, dtype=torch.float32, device=X.device)
        self.step += 1
        _check(lib.ch_mlp_train_step(_ptr(X, "X"), B, _ptr(label, "label"), _ptr(off, "off"), _ptr(mask, "mask"),
                                     ctypes.c_float(lam), _ptr(self.params, "params"), _ptr(self.master, "master"),
                                     _ptr(self.m, "m"), _ptr(self.v, "v"), self.step, ctypes.c_float(lr),
                                     _ptr(scratch, "scratch"), _ptr(loss, "loss"), _stream(stream)),
               "ch_mlp_train_step")
        return loss

    def train(self, X, label, off, mask, steps=400, batch=64, lr=3e-3, lam=1.0, seed=0):
        """Adam over random minibatches; returns the mean loss of each step."""
        import torch
        g = torch.Generator(device="cpu").manual_seed(seed)
        T = X.shape[0]
        B = min(batch, T)
        scratch = torch.empty(int(load().ch_mlp_scratch_floats(B)), dtype=torch.float32, device=X.device)
        loss = torch.empty(B, dtype=torch.float32, device=X.device)
        hist = []
        for _ in range(steps):
            pick = torch.randperm(T, generator=g)[:B].to(X.device)
            self.train_step(X[pick].contiguous(), label[pick].contiguous(), off[pick].contiguous(),
                            mask[pick].contiguous(), lam, lr, scratch, loss)
            hist.append(loss)
            loss = torch.empty_like(loss)
        return [float(h.mean()) for h in hist]


def time_hull_kgon(pts, dirs, ws, reps: int = 2) -> float:
    """ms of one ch_hull_kgon call (CUDA events, after one warm-up)."""
    import torch
    from . import ch_hull_kgon
    idx = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=pts.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)
    ch_hull_kgon(pts, dirs, idx, cnt, ws.buf)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ch_hull_kgon(pts, dirs, idx, cnt, ws.buf)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def time_hull_choice(pts, K, dirs, ws, reps: int = 2) -> float:
    """ms of one hull with the octagon and (K > 8) the K-gon over its
    survivors -- ch_hull_octagon_kgon, the pipeline ch_hull_learned runs
    for that choice (CUDA events, after one warm-up)."""
    import torch
    from . import ch_hull_octagon_kgon
    idx = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=pts.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=pts.device)

    def call():
        ch_hull_octagon_kgon(pts, dirs, K, None, idx, cnt, ws.buf)

    call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def make_labels(point_sets, ws, proposal: Proposal, candidates: int = 2, seed: int = 0, pipeline: str = "octagon"):
    """Training tensors from timings of the method itself: for every set,
    its features; label = the K whose best candidate polygon (no offsets, or
    one of ``candidates`` random offset vectors) gave the fastest hull; the
    offset target is that candidate's offsets (in units of pi / K).
    pipeline "octagon": the hull ch_hull_learned runs for each choice
    (K = 8: the octagon with the hull step's fan, i.e. ch_hull; K > 8: the
    K-gon over the octagon's survivors as well); "kgon": ch_hull_kgon (the
    K-gon alone, no fan)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    X, lab, off = [], [], []
    for p in point_sets:
        d = torch.from_numpy(np.ascontiguousarray(p, np.float32)).to(proposal.device)
        X.append(proposal.features(d).clone())
        best = (math.inf, 0, np.zeros(N_OFF))
        for ki, K in enumerate(KS):
            n_c = 0 if (pipeline == "octagon" and K == 8) else candidates
            cands = [np.zeros(K)] + [rng.uniform(-SPREAD, SPREAD, K) for _ in range(n_c)]
            for u in cands:
                dirs = torch.from_numpy(directions(K, u)).to(d.device)
                t = (time_hull_choice(d, K, dirs, ws) if pipeline == "octagon" else time_hull_kgon(d, dirs, ws))
                if t < best[0]:
                    pad = np.zeros(N_OFF)
                    pad[:K] = u
                    best = (t, ki, pad)
        lab.append(best[1])
        off.append(best[2])
        del d
    dev = proposal.device
    return (torch.stack(X), torch.tensor(lab, dtype=torch.int32, device=dev),
            torch.tensor(np.array(off), dtype=torch.float32, device=dev),
            torch.ones(len(lab), dtype=torch.float32, device=dev))


def save_params(proposal: Proposal, path: str, meta: dict) -> None:
    """The BF16 parameters (as their 16-bit patterns) and a description."""
    import json
    import torch
    bits = proposal.params.view(torch.int16).cpu().numpy().astype(np.uint16)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez_compressed(path, params=bits, meta=json.dumps(meta))


def load_params(path: str, device="cuda"):
    """(Proposal with the saved BF16 parameters, their description)."""
    import json
    import torch
    z = np.load(path)
    prop = Proposal(device=device)
    bits = torch.from_numpy(z["params"].astype(np.int16)).to(prop.device)
    assert bits.numel() == prop.n_params, "parameter count"
    prop.params = bits.view(torch.bfloat16)
    prop.master = prop.params.to(torch.float32)
    return prop, json.loads(str(z["meta"]))


def train_from_generated(families, sets_per_family: int, n: int, seed: int, steps: int = 800, batch: int = 64,
                         lr: float = 3e-3, lam: float = 0.5, device="cuda", log=None):
    """Generates the families' sets (pointgen), labels them by timing every
    choice through the method itself, trains the MLP; returns (Proposal,
    description)."""
    import time
    import torch
    import pointgen
    from . import Workspace
    t0 = time.perf_counter()
    prop = Proposal(device=device, seed=seed)
    ws = Workspace(n, device=device)
    Xs, labs, offs = [], [], []
    for k, kind in enumerate(families):
        for s in range(sets_per_family):
            p = pointgen.make_family(kind, n, seed=1_000_000 + 10_000 * k + s)
            X, lab, off, _ = make_labels([p], ws, prop, seed=seed + 7919 * k + s)
            Xs.append(X)
            labs.append(lab)
            offs.append(off)
            if log and (s + 1) % 100 == 0:
                log(f"{kind}: {s + 1} sets labelled, {time.perf_counter() - t0:.0f} s")
    X = torch.cat(Xs)
    label = torch.cat(labs)
    off = torch.cat(offs)
    mask = torch.ones(len(label), dtype=torch.float32, device=prop.device)
    label_s = time.perf_counter() - t0
    hist = prop.train(X, label, off, mask, steps=steps, batch=batch, lr=lr, lam=lam, seed=seed)
    counts = np.bincount(label.cpu().numpy(), minlength=4).tolist()
    meta = {"families": list(families), "sets_per_family": sets_per_family, "points_per_set": n,
            "label_counts_K8_16_32_64": counts, "steps": steps, "batch": batch, "lr": lr,
            "final_loss": round(float(np.mean(hist[-20:])), 4), "label_seconds": round(label_s, 1),
            "train_seconds": round(time.perf_counter() - t0 - label_s, 1),
            "labels": "fastest of ch_hull (K=8: octagon + fan) and ch_hull_octagon_kgon with K in 16, 32, 64 "
                      "(no offsets and 2 random offset vectors each)"}
    return prop, meta


DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposal.npz")


def main():
    import argparse
    import pointgen
    ap = argparse.ArgumentParser(description="train the learned proposal on generated sets and save its weights")
    ap.add_argument("--sets-per-family", type=int, default=400)
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    a = ap.parse_args()
    prop, meta = train_from_generated(pointgen.FAMILIES, a.sets_per_family, a.n, a.seed, steps=a.steps,
                                      log=lambda m: print(m, flush=True))
    save_params(prop, a.out, meta)
    print(meta, flush=True)


if __name__ == "__main__":
    main()
