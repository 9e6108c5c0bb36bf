"""Batched time steps (ipc_newton_step_envs, the paper's batched
environments of Sec. 5): every environment of a batch is a time step of its
own, and its result is bit for bit the one a context holding that
environment alone computes with the same parameters -- positions,
velocities, Newton / PCG / line-search counts and status -- over several
steps with contact, with a moving master, and when one environment of the
batch fails while the others go on."""
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


def _bits(a):
    return a.detach().cpu().numpy().view(np.int64)


def _envs(n_steps_list=(4, 6, 3, 5), nqs=(3, 4, 5, 4)):
    return [flat_press(nq=nq, n_steps=k) for nq, k in zip(nqs, n_steps_list)]


def _slices(parts):
    off, out = 0, []
    for p in parts:
        out.append(slice(off, off + p.X.shape[0]))
        off += p.X.shape[0]
    return out


def _moff(parts):
    off, out = 0, []
    for p in parts:
        out.append(slice(off, off + p.Y0.shape[0]))
        off += p.Y0.shape[0]
    return out


def _compare(B, parts, prec, n_steps, xm_path=None):
    batch = S.concat_envs(parts)
    sl, ml = _slices(parts), _moff(parts)
    cb = B.Context(batch, precision=prec)
    xb = torch.as_tensor(batch.X.copy(), device="cuda")
    vb = torch.as_tensor(batch.v_dirichlet.copy(), device="cuda")
    alone = []
    for p in parts:
        c = B.Context(p, precision=prec, params=batch.params)
        alone.append((c, torch.as_tensor(p.X.copy(), device="cuda"), torch.as_tensor(p.v_dirichlet.copy(),
                                                                                       device="cuda")))
    top_b = torch.as_tensor(batch.dirichlet.astype(bool), device="cuda")
    vd_b = torch.as_tensor(batch.v_dirichlet, device="cuda")
    statuses = []
    for step in range(n_steps):
        xm_b = None if xm_path is None else torch.as_tensor(xm_path(batch.Y0, step), device="cuda")
        r, per = cb.newton_step_envs(xb, vb, xm_next=xm_b)
        statuses.append([q["status"] for q in per])
        for e, (c, x, v) in enumerate(alone):
            xm = None if xm_b is None else xm_b[ml[e]].contiguous()
            ra = c.newton_step(x, v, xm_next=xm)
            assert ra["status"] == per[e]["status"], (step, e, ra, per[e])
            for k in ("newton_iters", "pcg_iters", "halvings", "residual", "res0", "alpha0", "last_alpha",
                      "energy", "pred_used"):
                assert ra[k] == per[e][k], (step, e, k, ra[k], per[e][k])
            np.testing.assert_array_equal(_bits(xb[sl[e]]), _bits(x), err_msg=f"x step {step} env {e}")
            np.testing.assert_array_equal(_bits(vb[sl[e]]), _bits(v), err_msg=f"v step {step} env {e}")
            top = torch.as_tensor(parts[e].dirichlet.astype(bool), device="cuda")
            v[top] = torch.as_tensor(parts[e].v_dirichlet, device="cuda")[top]
        vb[top_b] = vd_b[top_b]
    cb.close()
    for c, _, _ in alone:
        c.close()
    return statuses


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_step_equals_each_env_alone(B, prec):
    parts = _envs()
    st = _compare(B, parts, prec, n_steps=5)
    # the pads reach the master within the five steps: contact was active
    assert all(s == 0 for row in st for s in row), st


def test_batch_step_with_moving_master(B):
    # every master rises 2 um a step while the pads press down (in contact
    # from the fourth step)
    parts = _envs(n_steps_list=(8, 8, 10, 12))
    lift = lambda Y0, t: Y0 + np.array([0.0, 0.0, 2e-6 * (t + 1)])
    st = _compare(B, parts, "fp64", n_steps=5, xm_path=lift)
    assert all(s == 0 for row in st for s in row), st


def test_failed_env_leaves_others_untouched(B):
    parts = _envs()
    # environment 2's top face is driven 2 mm through its master in one step:
    # its Dirichlet motion is not admissible (status infeasible, state kept)
    bad = parts[2]
    top = bad.dirichlet.astype(bool)
    bad.v_dirichlet = np.zeros_like(bad.X)
    bad.v_dirichlet[top, 2] = -2e-3 / bad.params["h"]
    st = _compare(B, parts, "fp64", n_steps=2)
    for row in st:
        assert row[2] == B.STEP_INFEASIBLE and row[0] == row[1] == row[3] == 0
    # the batch call reports the failure, and the failed environment's
    # positions are those it started the step with
    batch = S.concat_envs(parts)
    cb = B.Context(batch, precision="fp64")
    x = torch.as_tensor(batch.X.copy(), device="cuda")
    v = torch.as_tensor(batch.v_dirichlet.copy(), device="cuda")
    r = cb.newton_step(x, v)
    assert r["status"] == B.STEP_INFEASIBLE
    s2 = _slices(parts)[2]
    np.testing.assert_array_equal(x[s2].cpu().numpy(), batch.X[s2])
    np.testing.assert_array_equal(v[s2].cpu().numpy(), batch.v_dirichlet[s2])
    cb.close()
