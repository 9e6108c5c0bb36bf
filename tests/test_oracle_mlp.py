"""Pins of the warm-start network's FP64 reference (oracle/mlp_oracle.py):
a hand-worked forward pass, central finite differences of the loss against
the chain-rule gradient, Adam's first-step closed form, and BF16 rounding on
values whose nearest BF16 neighbours are known."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def small_params(seed=3, scale=1.0):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    # non-zero biases so that every bias gradient path is exercised
    return [a.astype(np.float64) * scale if a.ndim == 2 else rng.normal(0, 0.1, a.shape) for a in p]


def test_forward_hand_worked():
    """One vertex, weights chosen so every layer is a scaled copy: f = e_0,
    W1 = 2 e_0 e_0^T, W2 = W3 = I (first unit), W4 = [1, 0, ...] in row 0;
    biases b1_0 = -0.5 (positive pre-activation 1.5), b2 = b3 = 0,
    b4 = (0, 7, -1): y = (1.5, 7, -1)."""
    W1 = np.zeros((256, 32)); W1[0, 0] = 2.0
    W2 = np.zeros((256, 256)); W2[0, 0] = 1.0
    W3 = W2.copy()
    W4 = np.zeros((3, 256)); W4[0, 0] = 1.0
    b1 = np.zeros(256); b1[0] = -0.5
    # a unit whose pre-activation is negative must be cut by the ReLU
    W1[1, 0] = -3.0; W2[0, 1] = 100.0
    b4 = np.array([0.0, 7.0, -1.0])
    f = np.zeros((1, 32)); f[0, 0] = 1.0
    y, _ = M.forward([W1, b1, W2, np.zeros(256), W3, np.zeros(256), W4, b4], f)
    np.testing.assert_array_equal(y, [[1.5, 7.0, -1.0]])


def test_loss_constant_output():
    p = small_params()
    p[6] = np.zeros_like(p[6])
    p[7] = np.array([0.5, -1.0, 2.0])
    rng = np.random.default_rng(0)
    f = rng.normal(size=(7, 32))
    t = rng.normal(size=(7, 3))
    m = np.array([1, 1, 0, 1, 1, 0, 1], dtype=float)
    ref = np.sum(m[:, None] * (p[7] - t) ** 2) / (3 * m.sum())
    assert M.loss(p, f, t, m) == pytest.approx(ref, rel=1e-14)


def test_gradient_central_differences():
    rng = np.random.default_rng(5)
    p = small_params(scale=1.0)
    n = 6
    f = rng.normal(size=(n, 32))
    t = rng.normal(size=(n, 3))
    m = np.array([1, 0, 1, 1, 1, 1], dtype=float)
    L, g = M.grads(p, f, t, m)
    assert L == pytest.approx(M.loss(p, f, t, m), rel=1e-14)
    for k, P in enumerate(p):
        idx = [np.unravel_index(i, P.shape) for i in rng.choice(P.size, min(P.size, 12), replace=False)]
        for ij in idx:
            h = 1e-6 * max(1.0, abs(P[ij]))
            q = [a.copy() for a in p]
            q[k][ij] += h
            lp = M.loss(q, f, t, m)
            q[k][ij] -= 2 * h
            lm = M.loss(q, f, t, m)
            fd = (lp - lm) / (2 * h)
            scale = np.abs(g[k]).max()
            assert abs(fd - g[k][ij]) <= 1e-6 * scale + 1e-8 * abs(fd), (k, ij, fd, g[k][ij])


def test_masked_vertices_do_not_contribute():
    rng = np.random.default_rng(6)
    p = small_params()
    f = rng.normal(size=(4, 32))
    t = rng.normal(size=(4, 3))
    m = np.array([1, 1, 0, 1], dtype=float)
    L1, g1 = M.grads(p, f, t, m)
    t2 = t.copy(); t2[2] += 100.0
    L2, g2 = M.grads(p, f, t2, m)
    assert L1 == L2
    for a, b in zip(g1, g2):
        np.testing.assert_array_equal(a, b)


def test_adam_first_step_closed_form():
    """With zero moments, bias-corrected step 1 moves each parameter by
    -lr g / (|g| + eps)."""
    rng = np.random.default_rng(8)
    p = [rng.normal(size=(4, 3)), rng.normal(size=5)]
    g = [rng.normal(size=(4, 3)), rng.normal(size=5)]
    z = [np.zeros_like(a) for a in p]
    newp, m1, m2 = M.adam_step(p, g, z, z, 1, lr=1e-3, eps=1e-8)
    for a, b, gi in zip(newp, p, g):
        np.testing.assert_allclose(a - b, -1e-3 * gi / (np.abs(gi) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1[0], 0.1 * g[0])
    np.testing.assert_allclose(m2[1], 0.001 * g[1] ** 2)


def test_bf16_round_known_values():
    one = 1.0
    vals = np.array([one, one + 2 ** -8, one + 3 * 2 ** -8, one + 2 ** -7, -2.5, 3.0e38, 1e-40],
                    dtype=np.float32)
    # 1 + 2^-8 ties to the even neighbour 1; 1 + 3 * 2^-8 ties to 1 + 2^-6
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5], dtype=np.float32)
    got = M.bf16_round(vals)
    np.testing.assert_array_equal(got[:5], want)
    # BF16 keeps the FP32 exponent range: large values stay finite
    assert np.isfinite(got[5]) and abs(got[5] / 3.0e38 - 1) < 2 ** -8
    # every result has its low 16 bits clear
    assert np.all((got.view(np.uint32) & 0xFFFF) == 0)


def test_features_definition():
    """The feature map's fixed points: zero displacement, velocity and force
    give zeros in those slots; the rest box maps onto [-1, 1] with its corners
    at the ends; sin^2 + cos^2 = 1 per frequency (to BF16 rounding); forces
    beyond 8 force_scale clamp; the contact flag follows the gradient rows."""
    from oracle import mlp_oracle as M
    rng = np.random.default_rng(0)
    X = rng.uniform(-1e-3, 2e-3, (50, 3))
    X[0] = X.min(axis=0)
    X[1] = X.max(axis=0)
    g = np.zeros((50, 3))
    g[5] = [1.0, -2.5e-4, 0.0]
    f = M.features(X, np.zeros_like(X), X, np.arange(50) % 2, np.arange(50) % 3 == 0, g,
                   1e-3, 1e-3, 1e-5, 1e-3)
    assert f.dtype == np.float32 and f.shape == (50, 32)
    assert np.all(f[:, 0:6] == 0.0)
    np.testing.assert_array_equal(f[0, 6:9], [-1, -1, -1])
    np.testing.assert_array_equal(f[1, 6:9], [1, 1, 1])
    assert np.all(np.abs(f[:, 6:9]) <= 1.0)
    np.testing.assert_array_equal(f[:, 9], np.arange(50) % 2)
    np.testing.assert_array_equal(f[:, 10], (np.arange(50) % 3 == 0))
    np.testing.assert_array_equal(f[5, 11:14], [-8.0, 0.25, 0.0])   # force = -g / 1e-3, clamped
    np.testing.assert_array_equal(f[:, 14], np.arange(50) == 5)
    s2c2 = f[:, 15:27:2].astype(np.float64) ** 2 + f[:, 16:27:2].astype(np.float64) ** 2
    np.testing.assert_allclose(s2c2, 1.0, atol=2e-2)
    assert np.all(f[:, 27:] == 0.0)
    # every value is a BF16 number
    np.testing.assert_array_equal(M.bf16_round(f), f)
