"""GPU checks of the learned proposal (mlp.cu through the C ABI) against the
numpy reference oracle/mlp.py: features bit for bit, the forward pass and
one training step within binary32-accumulation tolerance, training that
learns a separable task, and hulls with the proposed polygon equal to the
oracle's."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_10581_gb300 as ch
import pointgen
from oracle import mlp
from paper_2303_10581_gb300 import learned

pytestmark = pytest.mark.gpu


def dev(p):
    return torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()


@pytest.mark.parametrize("n", [1, 5, 4095, 4096, 4097, 100_003, 1_000_000])
@pytest.mark.parametrize("kind", pointgen.FAMILIES)
def test_features_bit_exact(kind, n):
    p = pointgen.make_family(kind, n, seed=n)
    f = learned.Proposal(seed=1).features(dev(p)).cpu().numpy()
    assert np.array_equal(f.view(np.uint32), mlp.features(p).view(np.uint32))


def params_f32(prop):
    return prop.params.float().cpu().numpy()


def test_forward_matches_reference():
    prop = learned.Proposal(seed=3)
    rng = np.random.default_rng(0)
    X = (rng.uniform(0, 1, (37, 1024)) / 40).astype(np.float32)
    out = prop.forward(dev(X)).cpu().numpy()
    _, _, ref = mlp.forward(X, params_f32(prop))
    assert np.allclose(out, ref, rtol=1e-4, atol=1e-5)


def test_train_step_matches_reference():
    prop = learned.Proposal(seed=4)
    rng = np.random.default_rng(1)
    B = 24
    X = (rng.uniform(0, 1, (B, 1024)) / 30).astype(np.float32)
    label = rng.integers(0, 4, B).astype(np.int32)
    off = rng.uniform(-0.4, 0.4, (B, 64)).astype(np.float32)
    mask = (rng.uniform(0, 1, B) > 0.25).astype(np.float32)
    p0, w0 = params_f32(prop), prop.master.cpu().numpy().astype(np.float64)
    loss = prop.train_step(dev(X), torch.from_numpy(label).cuda(), dev(off), dev(mask), lam=0.5, lr=1e-3)
    ref_loss, g = mlp.grads(X, p0, label, off, mask, 0.5)
    assert np.allclose(loss.cpu().numpy(), ref_loss, rtol=1e-4, atol=1e-5)
    w_ref, _, _ = mlp.adam(w0, g, np.zeros_like(w0), np.zeros_like(w0), 1, 1e-3)
    w = prop.master.cpu().numpy().astype(np.float64)
    bad = np.abs(w - w_ref) > 1e-6
    assert bad.mean() < 1e-3                    # near-zero gradients may differ in sign
    assert np.all(np.abs(w - w_ref) <= 2.1e-3)  # a step never exceeds lr per parameter
    # the kernels read the BF16 copy of the updated master weights
    assert np.array_equal(params_f32(prop), mlp.bf16_round(prop.master.cpu().numpy()))


def test_training_learns_the_family():
    prop = learned.Proposal(seed=5)
    X, y = [], []
    for k, kind in enumerate(pointgen.FAMILIES):
        for s in range(24):
            X.append(prop.features(dev(pointgen.make_family(kind, 50_000, seed=1000 * k + s))))
            y.append(k)
    X = torch.stack(X)
    label = torch.tensor(y, dtype=torch.int32, device="cuda")
    off = torch.zeros((len(y), 64), dtype=torch.float32, device="cuda")
    mask = torch.zeros(len(y), dtype=torch.float32, device="cuda")
    hist = prop.train(X, label, off, mask, steps=300, batch=48, lr=3e-3)
    assert np.mean(hist[-20:]) < 0.5 * np.mean(hist[:5])
    pred = prop.forward(X).cpu().numpy()[:, :4].argmax(1)
    assert (pred == np.array(y)).mean() >= 0.9


@pytest.mark.parametrize("kind", pointgen.FAMILIES)
def test_learned_hull_is_the_oracle_hull(kind):
    prop = learned.Proposal(seed=6)
    p = pointgen.make_family(kind, 300_003, seed=7)
    ws = ch.Workspace(len(p))
    idx, cnt, K = prop.hull(dev(p), ws)
    torch.cuda.synchronize()
    assert ch.ch_last_error(ws.buf) == ch.CH_OK
    assert K in learned.KS
    assert np.array_equal(idx[: int(cnt.item())].cpu().numpy().view(np.uint32), oracle.hull(p))
