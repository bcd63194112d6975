"""Pins of the numpy reference of the learned proposal (oracle/mlp.py): its
gradient against central finite differences of its own loss, the softmax
cross-entropy gradient's closed forms, BF16 rounding against exactly
representable cases, and the occupancy features on constructed inputs."""
import numpy as np
import pytest

from oracle import mlp


def small_problem(seed=0, B=5):
    rng = np.random.default_rng(seed)
    params = (rng.standard_normal(mlp.N_PARAMS) * 0.05).astype(np.float64)
    X = rng.uniform(0, 1, (B, mlp.IN)) / 50
    label = rng.integers(0, 4, B)
    off = rng.uniform(-0.4, 0.4, (B, 64))
    mask = (rng.uniform(0, 1, B) > 0.3).astype(np.float64)
    return params, X, label, off, mask


def test_gradient_matches_finite_differences():
    params, X, label, off, mask = small_problem()
    lam = 0.7
    _, g = mlp.grads(X, params, label, off, mask, lam)
    rng = np.random.default_rng(1)
    # parameters from every block (W1, b1, W2, b2, W3, b3)
    bounds = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    picks = np.concatenate([rng.integers(lo, hi, 6) for lo, hi in zip(bounds[:-1], bounds[1:])])
    h = 1e-6
    for i in picks:
        e = np.zeros_like(params)
        e[i] = h
        lp = mlp.grads(X, params + e, label, off, mask, lam)[0].mean()
        lm = mlp.grads(X, params - e, label, off, mask, lam)[0].mean()
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_cross_entropy_gradient_closed_forms():
    rng = np.random.default_rng(2)
    out = rng.standard_normal((7, mlp.OUT))
    label = rng.integers(0, 4, 7)
    loss, d = mlp.loss_grad(out, label, np.zeros((7, 64)), np.zeros(7), 1.0)
    assert np.allclose(d[:, :4].sum(1), 0.0)               # softmax minus one-hot sums to zero
    assert np.all(d[np.arange(7), label] < 0)
    assert np.allclose(d[:, 4:], 0.0)                        # no offset label: no offset gradient
    eq = np.zeros((1, mlp.OUT))
    l1, _ = mlp.loss_grad(eq, np.array([2]), np.zeros((1, 64)), np.zeros(1), 1.0)
    assert np.isclose(l1[0], np.log(4.0))                    # equal logits


def test_bf16_rounding():
    v = np.array([1.0, 1.5, -2.0, 3.140625, 0.0], np.float32)   # representable in BF16
    assert np.array_equal(mlp.bf16_round(v), v)
    one = np.float32(1.0)
    half_ulp = np.float32(2.0 ** -8)                              # BF16 spacing at 1 is 2^-7
    assert mlp.bf16_round(np.array([one + half_ulp], np.float32))[0] == one          # tie to even
    assert mlp.bf16_round(np.array([one + 3 * half_ulp], np.float32))[0] == np.float32(1 + 2 ** -6)  # tie to even


def test_features_constructed_inputs():
    same = np.full((10, 2), 3.0, np.float32)
    f = mlp.features(same)
    assert f[0] == 1.0 and f.sum() == 1.0                         # zero width: one cell
    corners = np.array([(0, 0), (1, 1)] * 50, np.float32)
    f = mlp.features(corners)
    assert f[0] == np.float32(0.5) and f[mlp.IN - 1] == np.float32(0.5)
    rng = np.random.default_rng(3)
    p = rng.standard_normal((100_000, 2)).astype(np.float32)
    f = mlp.features(p)
    assert abs(float(f.sum()) - 1.0) < 1e-5 and f.min() >= 0
    # the sample: evenly spaced indices, 4096 of them
    q = p.copy()
    q[1] = (100.0, 100.0)             # index 1 is not sampled (floor(j n / 4096) skips it)
    assert np.array_equal(mlp.features(q), f)


def test_adam_first_step_moves_by_lr():
    w, m, v = mlp.adam(np.zeros(3), np.array([2.0, -3.0, 0.5]), np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(w, [-0.01, 0.01, -0.01], atol=1e-9)   # bias-corrected: lr * sign(g)


def test_proposal_directions_match_the_input_generator():
    """The directions the learned proposal builds (offsets in units of
    pi / K) are the input generator's, bit for bit."""
    import pointgen
    from paper_2303_10581_gb300 import learned
    for K in learned.KS:
        u = np.random.default_rng(K).uniform(-0.4, 0.4, K)
        assert np.array_equal(learned.directions(K), pointgen.kgon_directions(K))
        assert np.array_equal(learned.directions(K, u), pointgen.kgon_directions(K, u * np.pi / K))
    assert np.array_equal(learned.directions(8), np.array(
        [[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1]], np.float32))
