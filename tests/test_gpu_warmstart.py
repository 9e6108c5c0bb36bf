"""GPU warm-start network (tcgen05 kernels through the C ABI) against the FP64
reference network in oracle/mlp_oracle.py.

The oracle is fed the same BF16-rounded (round to nearest even) weights
W1..W3 and features the GPU multiplies; the GPU additionally rounds the
hidden activations and back-propagated signals to BF16, which bounds the
agreement: forward output within 2e-2 (relative L2), loss within 2e-2,
every parameter gradient with cosine >= 0.999 and relative L2 <= 5e-2 for
batches of 1000+ vertices (0.99 and 1e-1 for a batch of 18, whose gradient
is a sum of too few terms for the BF16 rounding to average out).
Adam is compared exactly: the oracle's update applied to the GPU's own
gradient and parameters must reproduce the GPU's updated parameters to FP32
rounding.  Sizes span several 128-row tiles with a ragged tail and, for the
split-K weight gradient, more vertex chunks than SMs."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2605_24339_b300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24339_b300 import binding
    binding.lib()
    return binding


def scene_with(nq, nz):
    """A pad scene of (nq+1)^2 (nz+1) vertices (only its size matters here)."""
    return S.tactile_indent(n_quads=nq, side=nq * 0.5e-3, nz=nz, thick=nz * 0.25e-3, sphere_subdiv=1)


def flat(params):
    return np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in params])


def unflat(v):
    out, k = [], 0
    for (o, i) in M.SIZES:
        out.append(v[k:k + o * i].reshape(o, i)); k += o * i
        out.append(v[k:k + o]); k += o
    return out


def oracle_view(params):
    """The parameters as the GPU multiplies them: W1..W3 in BF16, W4 and the
    biases in FP32."""
    q = [np.asarray(p, dtype=np.float32) for p in params]
    for k in (0, 2, 4):
        q[k] = M.bf16_round(q[k])
    return [a.astype(np.float64) for a in q]


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def cosine(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def data(n, seed):
    rng = np.random.default_rng(seed)
    f = M.bf16_round(rng.normal(0, 1, (n, 32)).astype(np.float32))
    t = rng.normal(0, 1, (n, 3)).astype(np.float32)
    m = (rng.random(n) < 0.8).astype(np.float32)
    return f, t, m


SIZES = [(2, 1), (10, 8), (40, 11)]   # 18, 1089 and 20172 vertices


@pytest.mark.parametrize("nq,nz", SIZES)
def test_forward_matches_oracle(B, nq, nz):
    sc = scene_with(nq, nz)
    n = sc.X.shape[0]
    params = M.init_params(7)
    params[1][:] = np.random.default_rng(1).normal(0, 0.05, 256)
    ctx = B.Context(sc, precision="mixed")
    ctx.ws_create(flat(params))
    f, _, _ = data(n, 2)
    y = ctx.ws_forward(torch.as_tensor(f).to(torch.bfloat16).cuda()).cpu().numpy()
    yo, _ = M.forward(oracle_view(params), f)
    assert np.all(np.isfinite(y))
    assert rel(y, yo) < 2e-2
    ctx.close()


@pytest.mark.parametrize("nq,nz", SIZES)
def test_gradients_match_oracle(B, nq, nz):
    sc = scene_with(nq, nz)
    n = sc.X.shape[0]
    params = M.init_params(11)
    rng = np.random.default_rng(3)
    for k in (1, 3, 5, 7):
        params[k][:] = rng.normal(0, 0.05, params[k].shape)
    ctx = B.Context(sc, precision="mixed")
    ctx.ws_create(flat(params))
    f, t, m = data(n, 4)
    loss, g = ctx.ws_grads(torch.as_tensor(f).to(torch.bfloat16).cuda(), t, m)
    Lo, go = M.grads(oracle_view(params), f, t, m)
    assert loss == pytest.approx(Lo, rel=2e-2)
    cmin, rmax = (0.999, 5e-2) if n >= 1000 else (0.99, 1e-1)
    for k, (a, b) in enumerate(zip(unflat(g), go)):
        print(f"n={n} param {k}: cosine {cosine(a, b):.6f} rel {rel(a, b):.3e}")
        assert cosine(a, b) >= cmin, (k, cosine(a, b))
        assert rel(a, b) <= rmax, (k, rel(a, b))
    ctx.close()


def test_adam_step_matches_oracle(B):
    sc = scene_with(10, 8)
    n = sc.X.shape[0]
    params = M.init_params(13)
    ctx = B.Context(sc, precision="mixed")
    ctx.ws_create(flat(params), lr=1e-3)
    f, t, m = data(n, 5)
    ft = torch.as_tensor(f).to(torch.bfloat16).cuda()
    zeros = [np.zeros_like(p, dtype=np.float64) for p in params]
    p_cur = [p.astype(np.float64) for p in params]
    m1, m2 = zeros, [z.copy() for z in zeros]
    for step in range(1, 4):
        _, g = ctx.ws_grads(ft, t, m)
        ctx.ws_train_step(ft, t, m)
        p_cur, m1, m2 = M.adam_step(p_cur, [a.astype(np.float64) for a in unflat(g)], m1, m2, step, lr=1e-3)
        got = unflat(ctx.ws_params())
        for a, b in zip(got, p_cur):
            np.testing.assert_allclose(a, b, rtol=2e-6, atol=2e-6 * 1e-3)
        p_cur = [a.astype(np.float64) for a in got]   # follow the GPU's FP32 state
    ctx.close()


def test_training_reduces_loss(B):
    """A smooth target of the features: 150 Adam steps cut the loss well
    below its start."""
    sc = scene_with(10, 8)
    n = sc.X.shape[0]
    ctx = B.Context(sc, precision="mixed")
    ctx.ws_create(flat(M.init_params(17)), lr=2e-3)
    f, _, m = data(n, 6)
    t = np.stack([np.sin(f[:, 0]), 0.5 * f[:, 1] * f[:, 2], np.tanh(f[:, 3] - f[:, 4])], 1).astype(np.float32)
    ft = torch.as_tensor(f).to(torch.bfloat16).cuda()
    l0 = ctx.ws_train_step(ft, t, m)
    for _ in range(150):
        l1 = ctx.ws_train_step(ft, t, m)
    assert l1 < 0.2 * l0, (l0, l1)
    ctx.close()


def test_warmstart_deterministic(B):
    sc = scene_with(40, 11)
    n = sc.X.shape[0]
    f, t, m = data(n, 9)
    outs = []
    for _ in range(2):
        ctx = B.Context(sc, precision="mixed")
        ctx.ws_create(flat(M.init_params(19)))
        ft = torch.as_tensor(f).to(torch.bfloat16).cuda()
        for _ in range(2):
            ctx.ws_train_step(ft, t, m)
        outs.append((ctx.ws_params(), ctx.ws_forward(ft).cpu().numpy()))
        ctx.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
