"""Training pipeline of the learned warm start (network and kernels in
csrc/warmstart.cu, entry points ipc_ws_*).

The solver generates its own data: a rollout of time steps records, per step,
the features of (x^t, v^t) and the target
    (x^{t+1} - x^t - h v^t) / disp_scale
for every free vertex (Dirichlet vertices are masked out).  Training runs
Adam over the recorded steps with the project's tcgen05 forward and backward
kernels.  At run time ipc_ws_predict gives dx_pred = h v + disp_scale * y,
which ipc_newton_step admits only through its CCD-filtered start and only
when its residual is not worse than the plain predictor's.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

N_PARAM = 140803
LAYERS = [(256, 32), (256, 256), (256, 256), (3, 256)]


def init_params(seed: int) -> np.ndarray:
    """Flattened initial parameters: He-uniform weights (bound sqrt(6/fan_in))
    and zero biases, from a seeded PCG64 stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for (o, i) in LAYERS:
        b = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-b, b, size=o * i).astype(np.float32))
        parts.append(np.zeros(o, dtype=np.float32))
    out = np.concatenate(parts)
    assert out.size == N_PARAM
    return out


def default_scales(scene) -> dict:
    """Feature and target scales of a scene: positions in units of the mean
    slave edge, displacements in units of one step of the scripted
    (Dirichlet) motion, contact forces in units of kappa * edge^2 * dhat."""
    X = scene.X
    e = scene.stris
    lbar = float(np.mean(np.linalg.norm(X[e[:, 1]] - X[e[:, 0]], axis=1))) if e.shape[0] else 1e-3
    h = scene.params["h"]
    vmax = float(np.abs(scene.v_dirichlet).max()) if scene.v_dirichlet.size else 0.0
    disp = h * vmax if vmax > 0 else 1e-3 * lbar
    force = scene.params["kappa"] * lbar * lbar * scene.params["dhat"]
    return {"pos_scale": lbar, "disp_scale": disp, "force_scale": force}


@dataclass
class Sample:
    feats: object            # torch bfloat16 [n, 32] (device)
    target: object           # torch float32 [n, 3] (device)
    mask: object             # torch float32 [n] (device)


@dataclass
class Rollout:
    states: list = field(default_factory=list)     # (x, v) at the start of each step (device)
    samples: list = field(default_factory=list)    # training samples, one per step
    stats: list = field(default_factory=list)      # ipc_newton_step statistics


def rollout(ctx, scene, x, v, n_steps: int, xm=None, record: bool = True) -> Rollout:
    """Advance (x, v) in place by n_steps plain-predictor time steps, keeping
    every start state and, if record, the (features, target) pair of each
    step.  Dirichlet velocities are reset to the scene's script after each
    step.  Stops early at a step that does not converge."""
    import torch
    out = Rollout()
    top = torch.as_tensor(scene.dirichlet.astype(bool), device=x.device)
    vd = torch.as_tensor(scene.v_dirichlet, device=x.device, dtype=torch.float64)
    xm = torch.as_tensor(scene.Y0 if xm is None else xm, device=x.device, dtype=torch.float64)
    free = (~top).to(torch.float32)
    h = scene.params["h"]
    disp = ctx.ws_disp_scale if record else 1.0
    for _ in range(n_steps):
        x0, v0 = x.clone(), v.clone()
        out.states.append((x0, v0))
        f = ctx.ws_features(x0, v0, xm) if record else None
        st = ctx.newton_step(x, v)
        out.stats.append(st)
        if st["status"] != 0:
            break
        if record:
            tgt = ((x - x0 - h * v0) / disp).to(torch.float32)
            out.samples.append(Sample(f, tgt.contiguous(), free.clone()))
        v[top] = vd[top]
    return out


def train(ctx, samples, n_iters: int, seed: int = 0) -> list:
    """Adam over the recorded samples in a seeded random order; returns the
    loss of every iteration."""
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(n_iters):
        s = samples[int(rng.integers(len(samples)))]
        losses.append(ctx.ws_train_step(s.feats, s.target, s.mask))
    return losses


def compare_starts(ctx, scene, states, xm=None) -> dict:
    """Solve the step from every state twice, with the plain predictor and
    with the learned start; returns the Newton iterations and wall times."""
    import torch
    xm = torch.as_tensor(scene.Y0 if xm is None else xm, device=states[0][0].device, dtype=torch.float64)
    res = {"plain": [], "learned": []}
    for x0, v0 in states:
        for mode in ("plain", "learned"):
            xs, vs = x0.clone(), v0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dx = ctx.ws_predict(xs, vs, xm) if mode == "learned" else None
            st = ctx.newton_step(xs, vs, dx_pred=dx)
            torch.cuda.synchronize()
            st["wall_ms"] = (time.perf_counter() - t0) * 1e3
            res[mode].append(st)
    return res
