"""Time step with a deformable master (ipc_newton_step_joint; Sec. 4.2-4.3
with Eq. gap) against the oracle's joint step on the contact patch test
(Sec. 5.1): the same status, the same Newton iteration counts on the first
steps and positions within 1e-6 of the step's displacement in FP64 (3e-5
mixed; why not closer: see the comment of the parity test); the
patch test on the GPU (mean sigma_zz = -10 in both blocks to 2e-3, the
largest single-tet error bounded by the order of magnitude); bitwise
repeatable steps (the master rows and blocks are summed in a fixed order);
and a contact block outside the slave-master block pattern reported as
IPC_ERR_CAPACITY, not written."""
import numpy as np
import pytest

from helpers import patch_report
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


def _scene(newton_tol=1e-5, pcg_rel_tol=1e-3, **kw):
    sc, f = S.patch_test(kappa=kw.pop("kappa", 1e4), h=0.05, density=1.0, **kw)
    sc.params["newton_tol"] = newton_tol
    sc.params["pcg_rel_tol"] = pcg_rel_tol
    return sc, f


# The upper block is free sideways (only its inertia holds it), so the
# system is ill-conditioned and the last Newton iterations of a step sit at
# the noise floor of the sufficient-decrease test: the expected decrease
# there is below the rounding of the forces, so the oracle and the GPU (sums
# in other orders) may take a halving or an iteration more or less.  Both
# stop within the residual tolerance, so the steps are compared within
# 1e-6 (FP64; the first steps agree to ~1e-14) and 3e-5 (mixed) of the
# displacement, and the iteration counts on the first two steps only.  The
# mixed step stops at a residual of 1e-5 (the FP32 matrix reaches no
# lower on this system): two stopping points within that residual of the
# ill-conditioned lateral mode differ by ~1e-5 of the displacement (1.3e-5
# measured with the elastic terms in double-float).
@pytest.mark.parametrize("prec,tol,ntol,ptol", [("fp64", 1e-6, 1e-7, 1e-10), ("mixed", 3e-5, 1e-5, 1e-3)])
def test_joint_step_matches_oracle(B, oracle_mod, prec, tol, ntol, ptol):
    sc, f = _scene(newton_tol=ntol, pcg_rel_tol=ptol)
    sim = oracle_mod.Sim(oracle_mod.Scene(sc))
    sim.set_fext(f)
    ctx = B.Context(sc, precision=prec)
    ft = torch.as_tensor(f, device="cuda")
    x = np.concatenate([sc.X, sc.Y0])
    v = np.zeros_like(x)
    for step in range(6):
        xo, vo, st = sim.step(x, v)
        xg = torch.as_tensor(x, device="cuda").contiguous()
        vg = torch.as_tensor(v, device="cuda").contiguous()
        r = ctx.newton_step_joint(xg, vg, f_ext=ft)
        assert st.status == 0, (step, st.status)
        assert r["status"] == 0, (step, r)
        if prec == "fp64" and step < 2:   # before the noise floor is reached: the same iterations
            assert r["newton_iters"] == st.newton_iters
        d = np.linalg.norm(xo - x)
        assert d > 0
        assert np.linalg.norm(xg.cpu().numpy() - xo) <= tol * d, step
        assert np.abs(vg.cpu().numpy() - vo).max() <= tol * np.abs(vo).max() * 10, step
        x, v = xo, vo
    ctx.close()


def test_patch_test_gpu(B):
    sc, f = _scene()
    ctx = B.Context(sc, precision="mixed")
    x = torch.as_tensor(np.concatenate([sc.X, sc.Y0]), device="cuda")
    v = torch.zeros_like(x)
    ft = torch.as_tensor(f, device="cuda")
    for step in range(12):
        r = ctx.newton_step_joint(x, v, f_ext=ft)
        assert r["status"] in (0, B.STEP_NOT_CONVERGED), (step, r)
    assert r["status"] == 0
    rep = patch_report(sc, x.cpu().numpy())
    print("patch test (GPU, mixed, kappa 1e4):", rep)
    for blk in ("upper", "lower"):
        assert rep[blk]["mean"] == pytest.approx(-10.0, rel=2e-3)
        assert rep[blk]["max_rel_err"] < 0.1
    ctx.close()


def test_joint_step_is_deterministic(B):
    sc, f = _scene()
    outs = []
    for _ in range(2):
        ctx = B.Context(sc, precision="mixed")
        x = torch.as_tensor(np.concatenate([sc.X, sc.Y0]), device="cuda")
        v = torch.zeros_like(x)
        ft = torch.as_tensor(f, device="cuda")
        for _ in range(3):
            ctx.newton_step_joint(x, v, f_ext=ft)
        outs.append(x.cpu().numpy().view(np.int64).copy())
        ctx.close()
    np.testing.assert_array_equal(outs[0], outs[1])


def test_contact_outside_pattern_is_reported(B):
    sc, f = _scene()
    # a pattern radius far below the rest gap: no slave-master pair is in
    # the pattern, so the first contact block has no place
    ctx = B.Context(sc, precision="fp64", params={"joint_radius": 1e-9})
    x = torch.as_tensor(np.concatenate([sc.X, sc.Y0]), device="cuda")
    v = torch.zeros_like(x)
    ft = torch.as_tensor(f, device="cuda")
    with pytest.raises(B.GmcpError) as ei:
        for _ in range(3):
            ctx.newton_step_joint(x, v, f_ext=ft)
    assert ei.value.status == 5
    ctx.close()


def test_kinematic_step_refused_with_master_body(B):
    sc, f = _scene()
    ctx = B.Context(sc, precision="fp64")
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = torch.zeros_like(x)
    with pytest.raises(B.GmcpError):
        ctx.newton_step(x, v)
    ctx.close()
