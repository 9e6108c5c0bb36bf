"""What the trained warm-start network gains over the plain predictor on the
gel-on-terrain press (594,441 vertices).

Data: a plain-predictor rollout from rest; steps 8-21 (contact starts at
step 10) train the network, steps 22-27 are held out.  The output layer
starts at zero (the untrained network is the plain predictor) and the loss
weights contact-front vertices (|target| > 0.02 of a step, or in contact)
over the rest (0.01).  Checked on the held-out steps:
  - the predicted start is admitted (its residual is not worse than the
    plain start's) in most steps, and the CCD-admissible fraction alpha0 of
    the start rises on average: the prediction moves the contact front
    consistently with the obstacle, which the constant-velocity predictor
    drives into it;
  - every step converges to the Newton tolerance with either start.
Printed, not asserted: the held-out losses of the network and of the plain
predictor, and both starts' Newton iteration counts and wall times.  On this
workload the iteration count is governed by the step bounds inside Newton,
and the learned start does not lower it."""
import numpy as np
import pytest

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


def test_warm_start_gain_on_terrain_press(B):
    from paper_2605_24339_b300 import warmstart as WS
    sc = S.gel_on_terrain()
    sc.params.update(max_newton=60)
    ctx = B.Context(sc, precision="mixed")
    p0 = WS.init_params(0)
    p0[-3 - 3 * 256:] = 0.0
    ctx.ws_create(p0, lr=3e-4, **WS.default_scales(sc))
    x = torch.as_tensor(sc.X.copy()).cuda()
    v = torch.as_tensor(sc.v_dirichlet.copy()).cuda()
    WS.rollout(ctx, sc, x, v, 8, record=False)
    ro = WS.rollout(ctx, sc, x, v, 20, record=True)
    assert len(ro.samples) == 20
    for smp in ro.samples:
        big = (smp.target.abs().amax(dim=1) > 0.02).float()
        smp.mask = (smp.mask * (0.01 + big + smp.feats[:, 14].float())).contiguous()
    WS.train(ctx, ro.samples[:14], 1500, seed=1)
    held = ro.samples[14:20]
    net = [ctx.ws_grads(s.feats, s.target, s.mask)[0] for s in held]
    zero = [float((s.mask[:, None] * s.target ** 2).sum() / (3 * s.mask.sum())) for s in held]
    print("held-out loss: network", net, "plain", zero)
    res = WS.compare_starts(ctx, sc, ro.states[14:20])
    for k in ("plain", "learned"):
        print(k, "newton iters", [r["newton_iters"] for r in res[k]], "alpha0",
              [round(r["alpha0"], 3) for r in res[k]], "pred_used", [r["pred_used"] for r in res[k]],
              "ms", [round(r["wall_ms"]) for r in res[k]])
        assert all(r["status"] == 0 and r["residual"] <= sc.params["newton_tol"] for r in res[k])
    used = [r["pred_used"] for r in res["learned"]]
    assert sum(used) > len(used) / 2
    a_plain = np.mean([r["alpha0"] for r in res["plain"]])
    a_learn = np.mean([r["alpha0"] for r in res["learned"]])
    assert a_learn > a_plain
    ctx.close()
