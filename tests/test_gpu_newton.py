"""GPU time step (ipc_newton_step through the C ABI) against the oracle's
implicit-Euler step (problem statement of Sec. 2.1, contact potential of
Sec. 4.2 with frozen samples per iterate, step bound of Sec. 4.5).

Each step starts both sides from the same state (the oracle's previous
output), so differences do not accumulate.  Tolerances: FP64 path -- same
status and Newton iteration count, positions within 1e-10 of the step's
displacement (relative L2; the two sides differ only in summation order, so
the iterates agree far below the Newton tolerance -- measured <= 1e-12);
mixed path (FP32 contact gradient and Hessian) -- converged, positions within
1e-7 of the displacement (measured <= 2e-10)."""
import numpy as np
import pytest

from helpers import flat_press
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


def sphere_press():
    sc = S.tactile_indent(n_quads=8, side=4e-3, nz=2, thick=1e-3, sphere_subdiv=3, radius=5e-3,
                          press=0.2e-3, n_steps=6)
    sc.params.update(pcg_rel_tol=1e-6)
    return sc


CASES = {"flat": (flat_press, 4), "sphere": (sphere_press, 3)}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_disp(xg, xo, x0):
    d = np.linalg.norm(xo - x0)
    return np.linalg.norm(xg - xo) / d if d > 0 else np.linalg.norm(xg - xo)


def run_compare(B, oracle_mod, sc, n_steps, precision, tol, same_iters, xm_path=None, pred=None):
    O = oracle_mod.Scene(sc)
    sim = oracle_mod.Sim(O)
    ctx = B.Context(sc, precision=precision)
    top = sc.dirichlet.astype(bool)
    x = sc.X.copy()
    v = sc.v_dirichlet.copy()
    worst = 0.0
    for step in range(n_steps):
        xm_next = None if xm_path is None else xm_path(step)
        dxp = None if pred is None else pred(x, v)
        xo, vo, st = sim.step(x, v, xm_next=xm_next, dx_pred=dxp)
        xg, vg = dev(x), dev(v)
        r = ctx.newton_step(xg, vg, xm_next=xm_next, dx_pred=dxp)
        assert st.status == 0 and r["status"] == 0, (step, st.status, r)
        assert r["residual"] <= sc.params["newton_tol"]
        if same_iters:
            assert r["newton_iters"] == st.newton_iters, (step, r["newton_iters"], st.newton_iters)
        e = rel_disp(xg.cpu().numpy(), xo, x)
        worst = max(worst, e)
        assert e < tol, (step, e)
        assert rel_disp(vg.cpu().numpy(), vo, v) < tol * 10
        np.testing.assert_array_equal(xg.cpu().numpy()[top], xo[top])
        x, v = xo, vo.copy()
        v[top] = sc.v_dirichlet[top]
    ctx.close()
    return worst


@pytest.mark.parametrize("case", ["flat", "sphere"])
def test_newton_step_fp64_matches_oracle(B, oracle_mod, case):
    make, n = CASES[case]
    run_compare(B, oracle_mod, make(), n, "fp64", 1e-10, True)


@pytest.mark.parametrize("case", ["flat", "sphere"])
def test_newton_step_mixed_converges_to_oracle(B, oracle_mod, case):
    make, n = CASES[case]
    run_compare(B, oracle_mod, make(), n, "mixed", 1e-7, False)


def test_newton_learned_start_matches_oracle(B, oracle_mod):
    """dx_pred start (Sec. 8 warm start): the predictor overshoots the plain
    one by 30 %, so the CCD-filtered start differs from x + h v."""
    sc = flat_press()
    run_compare(B, oracle_mod, sc, 3, "fp64", 1e-10, True,
                pred=lambda x, v: 1.3 * sc.params["h"] * v)


def test_newton_master_motion_matches_oracle(B, oracle_mod):
    """Master moving toward the pad while the top face is driven down (two
    steps, before the gap closes: a master motion that the additive CCD does
    not admit with the pad held at x^t makes the step infeasible, on both
    sides)."""
    sc = flat_press()
    Y0 = sc.Y0.copy()
    run_compare(B, oracle_mod, sc, 2, "fp64", 1e-10, True,
                xm_path=lambda k: Y0 + np.array([0.0, 0.0, 2e-5 * (k + 1)]))


def test_newton_zero_motion_is_stationary(B):
    sc = sphere_press()
    ctx = B.Context(sc, precision="fp64")
    x, v = dev(sc.X), dev(np.zeros_like(sc.X))
    r = ctx.newton_step(x, v)
    assert r["status"] == 0 and r["newton_iters"] <= 1
    np.testing.assert_allclose(x.cpu().numpy(), sc.X, rtol=0, atol=1e-14)
    ctx.close()


def test_newton_infeasible_master_motion_restores_state(B, oracle_mod):
    """A master jump through the pad is rejected by the CCD check before any
    Newton iteration; x and v are left at x^t, v^t (as in the oracle)."""
    sc = flat_press()
    xm_next = sc.Y0 + np.array([0.0, 0.0, 1.0e-3])
    O = oracle_mod.Scene(sc)
    _, _, st = oracle_mod.Sim(O).step(sc.X, sc.v_dirichlet, xm_next=xm_next)
    assert st.status == 3
    ctx = B.Context(sc, precision="fp64")
    x, v = dev(sc.X), dev(sc.v_dirichlet)
    r = ctx.newton_step(x, v, xm_next=xm_next)
    assert r["status"] == B.STEP_INFEASIBLE
    np.testing.assert_array_equal(x.cpu().numpy(), sc.X)
    np.testing.assert_array_equal(v.cpu().numpy(), sc.v_dirichlet)
    ctx.close()


def test_newton_step_deterministic(B):
    sc = sphere_press()
    outs = []
    for _ in range(2):
        ctx = B.Context(sc, precision="fp64")
        x, v = dev(sc.X), dev(sc.v_dirichlet)
        for _ in range(2):
            ctx.newton_step(x, v)
        outs.append(x.cpu().numpy())
        ctx.close()
    np.testing.assert_array_equal(outs[0], outs[1])


def test_config1_indent_converging_steps_match_oracle(B, oracle_mod):
    """The single-environment indent at its specified size (32x32-quad pad,
    4 tet layers, subdivision-3 icosphere, dhat 1e-4, kappa 1e5, h 1 ms,
    jitter 1e-5 m): its first four steps, which the oracle converges, on the
    GPU from the oracle's previous state each time.  FP64: same status and
    Newton iteration count, positions within 1e-10 of the step's
    displacement; mixed: converged, within 1e-7.  (The fifth step locks in
    both, on a primitive pair no sample covers near the indenter's tip.)"""
    sc = S.tactile_indent()
    O = oracle_mod.Scene(sc)
    sim = oracle_mod.Sim(O)
    ctx = {p: B.Context(sc, precision=p) for p in ("fp64", "mixed")}
    top = sc.dirichlet.astype(bool)
    x = sc.X.copy()
    v = sc.v_dirichlet.copy()
    iters = []
    for step in range(4):
        xo, vo, st = sim.step(x, v)
        assert st.status == 0, (step, st.status)
        iters.append(st.newton_iters)
        for prec, tol in (("fp64", 1e-10), ("mixed", 1e-7)):
            xg, vg = dev(x), dev(v)
            r = ctx[prec].newton_step(xg, vg)
            assert r["status"] == 0 and r["residual"] <= sc.params["newton_tol"], (prec, step, r)
            if prec == "fp64":
                assert r["newton_iters"] == st.newton_iters, (step, r["newton_iters"], st.newton_iters)
            e = rel_disp(xg.cpu().numpy(), xo, x)
            assert e < tol, (prec, step, e)
            np.testing.assert_array_equal(xg.cpu().numpy()[top], xo[top])
        x, v = xo, vo.copy()
        v[top] = sc.v_dirichlet[top]
    print("config 1 oracle Newton iterations, steps 0-3:", iters)
    for c in ctx.values():
        c.close()
