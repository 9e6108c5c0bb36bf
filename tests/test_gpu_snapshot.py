"""Checkpoint and resume (ipc_save / ipc_load): a context created from the
same scene and parameters and loaded from a snapshot continues bit for bit
as the context that wrote it -- positions, velocities, the moving master,
the step count and, with a learned warm start, the network and its Adam
state.  Corrupt or mismatched files are refused and change nothing."""
import numpy as np
import pytest

from helpers import flat_press
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24339_b300 import binding
    binding.lib()
    return binding


def _flat(params):
    return np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in params])


def _steps(ctx, sc, x, v, k, xm_path=None, t0=0, learned=False):
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    vd = torch.as_tensor(sc.v_dirichlet, device="cuda")
    for i in range(k):
        xm = None if xm_path is None else xm_path(t0 + i)
        dxp = ctx.ws_predict(x, v, xm if xm is not None else torch.as_tensor(sc.Y0, device="cuda")) \
            if learned else None
        r = ctx.newton_step(x, v, xm_next=xm, dx_pred=dxp)
        assert r["status"] == 0, r
        v[top] = vd[top]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_is_bitwise(B, tmp_path, prec):
    # the master rises 2 um a step while the top face presses the pad onto it
    # (in contact from the fourth step; the oracle converges on all five)
    sc = flat_press(nq=4, n_steps=8)
    lift = lambda t: sc.Y0 + np.array([0.0, 0.0, 2e-6 * (t + 1)])
    path = str(tmp_path / "snap.bin")
    a = B.Context(sc, precision=prec)
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = torch.as_tensor(sc.v_dirichlet.copy(), device="cuda")
    _steps(a, sc, x, v, 2, lift, 0)
    a.save(path, x, v)
    _steps(a, sc, x, v, 3, lift, 2)
    b = B.Context(sc, precision=prec)
    xb = torch.zeros_like(x)
    vb = torch.zeros_like(v)
    assert b.load(path, xb, vb) == 2
    _steps(b, sc, xb, vb, 3, lift, 2)
    assert torch.equal(x, xb) and torch.equal(v, vb)
    # the loaded master pose is the one the next step moves from: with the
    # rest pose instead, the master motion of step 5 would differ
    a.close()
    b.close()


def test_resume_with_network_is_bitwise(B, tmp_path):
    sc = flat_press(nq=4, n_steps=8)
    path = str(tmp_path / "snap_ws.bin")
    n = sc.X.shape[0]
    rng = np.random.default_rng(2)
    f = torch.as_tensor(M.bf16_round(rng.normal(0, 1, (n, 32)).astype(np.float32))).to(torch.bfloat16).cuda()
    t = torch.as_tensor(rng.normal(0, 1e-2, (n, 3)).astype(np.float32)).cuda()
    m = torch.ones(n, device="cuda")
    p0 = _flat(M.init_params(5))
    a = B.Context(sc, precision="mixed")
    a.ws_create(p0, lr=1e-3)
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = torch.as_tensor(sc.v_dirichlet.copy(), device="cuda")
    for _ in range(3):
        a.ws_train_step(f, t, m)
    _steps(a, sc, x, v, 1, learned=True)
    a.save(path, x, v)
    for _ in range(2):
        a.ws_train_step(f, t, m)
    _steps(a, sc, x, v, 2, learned=True)
    b = B.Context(sc, precision="mixed")        # no network yet: the snapshot creates it
    xb, vb = torch.zeros_like(x), torch.zeros_like(v)
    assert b.load(path, xb, vb) == 1
    for _ in range(2):
        b.ws_train_step(f, t, m)
    _steps(b, sc, xb, vb, 2, learned=True)
    np.testing.assert_array_equal(a.ws_params(), b.ws_params())
    assert torch.equal(x, xb) and torch.equal(v, vb)
    a.close()
    b.close()


def test_bad_snapshots_are_refused(B, tmp_path):
    sc = flat_press(nq=4, n_steps=4)
    a = B.Context(sc, precision="fp64")
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = torch.as_tensor(sc.v_dirichlet.copy(), device="cuda")
    path = tmp_path / "s.bin"
    a.save(str(path), x, v)
    raw = bytearray(path.read_bytes())
    xb = torch.full_like(x, 7.0)
    vb = torch.full_like(v, 7.0)
    for name, data in [("flipped", raw[:200] + bytes([raw[200] ^ 1]) + raw[201:]),
                       ("truncated", raw[:-16]), ("empty", b""),
                       ("version", raw[:8] + b"\x02" + raw[9:])]:
        bad = tmp_path / f"{name}.bin"
        bad.write_bytes(bytes(data))
        with pytest.raises(B.GmcpError):
            a.load(str(bad), xb, vb)
        assert float(xb.min()) == 7.0 and float(vb.max()) == 7.0   # untouched
    with pytest.raises(B.GmcpError):
        a.load(str(tmp_path / "missing.bin"), xb, vb)
    # a scene of other sizes
    other = flat_press(nq=3, n_steps=4)
    c = B.Context(other, precision="fp64")
    xo = torch.zeros((other.X.shape[0], 3), dtype=torch.float64, device="cuda")
    with pytest.raises(B.GmcpError):
        c.load(str(path), xo, torch.zeros_like(xo))
    a.close()
    c.close()
