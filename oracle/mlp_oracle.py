"""FP64 reference of the learned warm start's network (test infrastructure
only: the product never imports this module).

The network maps 32 per-vertex features to a 3-vector, the correction of the
plain predictor (x^{t+1} = x^t + h v^t + correction), through four affine
layers with ReLU between them:

    z1 = f W1^T + b1,  h1 = max(z1, 0)        W1: 256 x 32
    z2 = h1 W2^T + b2, h2 = max(z2, 0)        W2: 256 x 256
    z3 = h2 W3^T + b3, h3 = max(z3, 0)        W3: 256 x 256
    y  = h3 W4^T + b4                         W4:   3 x 256

Loss (per batch): L = sum_{v,c} m_v (y_vc - t_vc)^2 / (3 sum_v m_v), with a
per-vertex mask m (1 for vertices that count).  Training uses Adam (Kingma,
Ba 2015) with bias correction.  Every function below is the plain definition
with numpy matrix products in FP64.  "parity unpinned" applies to nothing
here: the gradient is pinned by central finite differences and Adam by its
first-step closed form (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

SIZES = [(256, 32), (256, 256), (256, 256), (3, 256)]


def init_params(seed: int):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from a
    seeded PCG64 stream.  Returns [W1, b1, W2, b2, W3, b3, W4, b4] (FP32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for (o, i) in SIZES:
        bound = np.sqrt(6.0 / i)
        out.append(rng.uniform(-bound, bound, size=(o, i)).astype(np.float32))
        out.append(np.zeros(o, dtype=np.float32))
    return out


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def forward(params, f):
    """Activations of every layer: returns (y, cache) in FP64."""
    W1, b1, W2, b2, W3, b3, W4, b4 = [np.asarray(p, dtype=np.float64) for p in params]
    f = np.asarray(f, dtype=np.float64)
    z1 = f @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + b3
    h3 = np.maximum(z3, 0.0)
    y = h3 @ W4.T + b4
    return y, (f, z1, h1, z2, h2, z3, h3)


def loss(params, f, t, m):
    y, _ = forward(params, f)
    m = np.asarray(m, dtype=np.float64)
    return float(np.sum(m[:, None] * (y - t) ** 2) / (3.0 * np.sum(m)))


def grads(params, f, t, m):
    """(loss, [dW1, db1, dW2, db2, dW3, db3, dW4, db4]) by the chain rule."""
    W1, b1, W2, b2, W3, b3, W4, b4 = [np.asarray(p, dtype=np.float64) for p in params]
    y, (f, z1, h1, z2, h2, z3, h3) = forward(params, f)
    m = np.asarray(m, dtype=np.float64)
    den = 3.0 * np.sum(m)
    L = float(np.sum(m[:, None] * (y - t) ** 2) / den)
    dy = 2.0 * m[:, None] * (y - t) / den
    dW4 = dy.T @ h3
    db4 = dy.sum(axis=0)
    dz3 = (dy @ W4) * (z3 > 0)
    dW3 = dz3.T @ h2
    db3 = dz3.sum(axis=0)
    dz2 = (dz3 @ W3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ f
    db1 = dz1.sum(axis=0)
    return L, [dW1, db1, dW2, db2, dW3, db3, dW4, db4]


def adam_step(params, g, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (params, m1, m2)."""
    newp, n1, n2 = [], [], []
    for p, gi, a, b in zip(params, g, m1, m2):
        a = beta1 * a + (1.0 - beta1) * gi
        b = beta2 * b + (1.0 - beta2) * gi * gi
        ah = a / (1.0 - beta1 ** step)
        bh = b / (1.0 - beta2 ** step)
        newp.append(p - lr * ah / (np.sqrt(bh) + eps))
        n1.append(a)
        n2.append(b)
    return newp, n1, n2


def features(x, v, X, dirichlet, surface, contact_grad, h, pos_scale, disp_scale, force_scale):
    """Per-vertex input features of the warm-start network (the project's own
    design; the paper has no learned component), FP64 then rounded to BF16:

      0-2   (x - X) / pos_scale
      3-5   h v / disp_scale
      6-8   Xn = 2 (X - lo) / (hi - lo) - 1, lo/hi the pad's rest box per axis
      9     Dirichlet flag
      10    slave-surface flag
      11-13 contact force -grad Psi / force_scale, clamped to [-8, 8]
      14    1 where the contact gradient row is nonzero
      15-26 per axis c: sin(pi Xn_c), cos(pi Xn_c), sin(2 pi Xn_c), cos(2 pi Xn_c)
      27-31 zero
    Returns FP32 values that are exactly BF16-representable, [n][32]."""
    x, v, X = (np.asarray(a, dtype=np.float64) for a in (x, v, X))
    g = np.asarray(contact_grad, dtype=np.float64)
    n = X.shape[0]
    f = np.zeros((n, 32))
    lo, hi = X.min(axis=0), X.max(axis=0)
    ext = np.where(hi > lo, hi - lo, 1.0)
    xn = 2.0 * (X - lo) / ext - 1.0
    f[:, 0:3] = (x - X) / pos_scale
    f[:, 3:6] = h * v / disp_scale
    f[:, 6:9] = xn
    f[:, 9] = np.asarray(dirichlet) != 0
    f[:, 10] = np.asarray(surface) != 0
    f[:, 11:14] = np.clip(-g / force_scale, -8.0, 8.0)
    f[:, 14] = np.any(g != 0.0, axis=1)
    for c in range(3):
        for k in (1, 2):
            col = 15 + 4 * c + 2 * (k - 1)
            f[:, col] = np.sin(np.pi * k * xn[:, c])
            f[:, col + 1] = np.cos(np.pi * k * xn[:, c])
    return bf16_round(f.astype(np.float32))
