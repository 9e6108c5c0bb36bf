"""The contact pass and the time step with the paper's clipped-overlap face
samples (Sec. 4.1 "Face samples", ipc_params.face_sampler = 1) against the
oracle in the same mode: face candidates (box-box within dhat) bit-exact;
FP64 path 1e-12 on energy, gradient and every Hessian block, mixed path
1e-5 / 1e-5 / 1e-4; the partial-overlap closed form of
tests/test_oracle_clip_mode.py; the implicit-Euler step with the same
Newton iteration counts and positions within 1e-10 of the displacement
(FP64)."""
import numpy as np
import pytest

from helpers import (MM, face_master, flat_press, hess_blocks_check, one_slave_triangle, rel, small_indent)
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


def _clip(sc):
    sc.params["face_sampler"] = 1
    return sc


def _scenes():
    out = []
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.12e-3, L=1)
    out.append(("indent", _clip(sc), x))
    parts, xs = [], []
    for k, (nq, press) in enumerate([(6, 0.08e-3), (9, 0.15e-3), (4, 0.05e-3)]):
        s, xx = small_indent(n_quads=nq, subdiv=2 + (k % 2), press=press, seed=20 + k)
        parts.append(s)
        xs.append(xx)
    out.append(("batch3", _clip(S.concat_envs(parts)), np.concatenate(xs)))
    return out


SCENES = _scenes()


@pytest.mark.parametrize("prec,tol,tol_h", [("fp64", 1e-12, 1e-12), ("mixed", 1e-5, 1e-4)])
@pytest.mark.parametrize("name,sc,x", SCENES, ids=[s[0] for s in SCENES])
def test_clip_mode_pass_parity(B, oracle_mod, name, sc, x, prec, tol, tol_h):
    ctx = B.Context(sc, precision=prec)
    O = oracle_mod.Scene(sc)
    try:
        r = ctx.barrier_eval(x, sc.Y0)
        o = O.contact(x, sc.Y0)
        for kind in range(3):
            np.testing.assert_array_equal(ctx.candidate_pairs(kind), O.candidates(kind, x, sc.Y0))
        assert o["energy"] > 0
        c = r["counts"]
        assert (c["point"], c["edge"], c["face"]) == tuple(int(v) for v in o["n_samples"])
        assert r["energy"] == pytest.approx(o["energy"], rel=tol)
        assert rel(r["grad"].double().cpu().numpy(), o["grad"]) < tol
        hess_blocks_check(r["hess"], o, tol_h)
        # the step bound in the same mode (FP64 in both precisions)
        rng = np.random.default_rng(2)
        dx = np.zeros_like(x)
        dx[:, 2] = -(1e-5 + 2e-5 * rng.random(x.shape[0]))
        g = ctx.ccd_max_step(x, dx, sc.Y0)
        a, al, aa = O.ccd_max_step(x, dx, sc.Y0)
        assert g["alpha_accd"] == aa
        assert g["alpha"] <= a and g["alpha"] == pytest.approx(a, rel=1e-9)
    finally:
        ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_clip_mode_partial_overlap_closed_form(B, prec, tol):
    g = 3e-5
    Y, F = face_master(g)
    sc, x, xm = one_slave_triangle(Y, F, kappa_edge=0.0, kappa_point=0.0)
    sc.params.update(face_sampler=1, delta_T=1e-9)
    ctx = B.Context(sc, precision=prec)
    try:
        r = ctx.barrier_eval(x, xm)
        d = g - sc.params["dhat"]
        E = sc.params["kappa"] * 0.5 * 0.82 ** 2 * MM * MM * (-d * d * np.log(g / sc.params["dhat"]))
        assert r["energy"] == pytest.approx(E, rel=tol)
    finally:
        ctx.close()


def test_clip_mode_newton_steps(B, oracle_mod):
    sc = _clip(flat_press(nq=4, n_steps=4))
    O = oracle_mod.Scene(sc)
    sim = oracle_mod.Sim(O)
    top = sc.dirichlet.astype(bool)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-7)):
        ctx = B.Context(sc, precision=prec)
        x, v = sc.X.copy(), sc.v_dirichlet.copy()
        for step in range(4):
            xo, vo, st = sim.step(x, v)
            xg = torch.as_tensor(x).cuda()
            vg = torch.as_tensor(v).cuda()
            r = ctx.newton_step(xg, vg)
            assert st.status == 0 and r["status"] == 0, (step, st.status, r)
            if prec == "fp64":
                assert r["newton_iters"] == st.newton_iters
            d = np.linalg.norm(xo - x)
            assert np.linalg.norm(xg.cpu().numpy() - xo) <= tol * d, step
            x, v = xo, vo.copy()
            v[top] = sc.v_dirichlet[top]
        ctx.close()
