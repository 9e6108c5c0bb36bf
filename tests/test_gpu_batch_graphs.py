"""Batching, CUDA graphs and the autotuner (all through the C ABI).

- A contact pass replayed from a captured CUDA graph gives bitwise the same
  energy, gradient, Hessian and step bound as plain launches, also after the
  positions change in place (the graph reads them through the same pointers).
- Every launch shape the autotuner may pick gives bitwise identical results.
- A batch of environments equals its environments evaluated one by one:
  gradient rows and step bounds bitwise, the energy to summation order
  (pairs never cross environments).
- The time step with graph-captured PCG chunks equals the plain one bitwise."""
import numpy as np
import pytest

from helpers import small_indent
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def pass_outputs(ctx, x, xm, dx):
    r = ctx.contact_pass(x, xm, dx, grad=True, hess=True, counts=True)
    return (r["energy"], r["grad"].cpu().numpy().copy(), r["hess"][2].cpu().numpy().copy(),
            r["alpha"], r["alpha_lin"], r["alpha_accd"], r["counts"]["face"])


def same(a, b):
    assert a[0] == b[0] and a[3:] == b[3:]
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])


def workload(seed=4):
    sc, x = small_indent(n_quads=12, subdiv=3, press=0.12e-3, L=2, seed=seed)
    rng = np.random.default_rng(seed)
    dx = np.zeros_like(x)
    dx[:, 2] = -(1e-5 + 2e-5 * rng.random(x.shape[0]))
    return sc, x, dx


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_is_bitwise_identical(B, prec):
    sc, x_np, dx_np = workload()
    plain = B.Context(sc, precision=prec, params={"use_graphs": 0})
    graph = B.Context(sc, precision=prec, params={"use_graphs": 1})
    x, xm, dx = dev(x_np), dev(sc.Y0), dev(dx_np)
    ref = pass_outputs(plain, x, xm, dx)
    for _ in range(3):                      # capture on the first call, then replays
        same(pass_outputs(graph, x, xm, dx), ref)
    # new positions in the same buffer: the replay must see them
    x.add_(torch.as_tensor(1e-6 * np.random.default_rng(1).normal(size=x_np.shape)).cuda())
    ref2 = pass_outputs(plain, x, xm, dx)
    same(pass_outputs(graph, x, xm, dx), ref2)
    assert ref2[0] != ref[0]
    plain.close(); graph.close()


def test_launch_shapes_do_not_change_results(B):
    sc, x_np, dx_np = workload(seed=7)
    ctx = B.Context(sc, precision="mixed")
    x, xm, dx = dev(x_np), dev(sc.Y0), dev(dx_np)
    ref = pass_outputs(ctx, x, xm, dx)
    for s_b, q_b in [(1, 2), (16, 32), (4, 8), (2, 16)]:
        ctx.set_launch_shape(s_b, q_b)
        same(pass_outputs(ctx, x, xm, dx), ref)
    s_b, q_b, ms = ctx.autotune(x, xm, dx, reps=2)
    assert s_b in (1, 2, 4, 8, 16) and q_b in (2, 4, 8, 16, 32) and ms > 0
    same(pass_outputs(ctx, x, xm, dx), ref)
    ctx.close()


def test_batch_equals_environments_one_by_one(B):
    parts, xs = [], []
    for k, (nq, press) in enumerate([(6, 0.08e-3), (9, 0.15e-3), (4, 0.05e-3), (8, 0.1e-3)]):
        s, xx = small_indent(n_quads=nq, subdiv=2 + (k % 2), press=press, seed=30 + k)
        parts.append(s)
        xs.append(xx)
    batch = S.concat_envs(parts)
    xb = np.concatenate(xs)
    rng = np.random.default_rng(2)
    dxs = [np.concatenate([1e-6 * rng.normal(size=(x.shape[0], 2)), -(1e-5 + 1e-5 * rng.random((x.shape[0], 1)))], 1)
           for x in xs]
    ctx = B.Context(batch, precision="fp64")
    eb, gb, _, ab, alb, aab, _ = pass_outputs(ctx, dev(xb), dev(batch.Y0), dev(np.concatenate(dxs)))
    ctx.close()
    e_sum, alphas, lins, accds, off = 0.0, [], [], [], 0
    for s, x, d in zip(parts, xs, dxs):
        # the batch carries one parameter set (kappa_edge / kappa_point come
        # from a scene's mean edge length): evaluate each env with it
        c = B.Context(s, precision="fp64", params=batch.params)
        e, g, _, a, al, aa, _ = pass_outputs(c, dev(x), dev(s.Y0), dev(d))
        c.close()
        np.testing.assert_array_equal(gb[off:off + x.shape[0]], g)
        off += x.shape[0]
        e_sum += e
        alphas.append(a); lins.append(al); accds.append(aa)
    assert eb == pytest.approx(e_sum, rel=1e-12)
    assert aab == min(accds)
    assert alb == min(lins)
    assert ab == min(alphas)


def test_newton_step_with_pcg_graphs_is_bitwise_identical(B):
    from helpers import flat_press
    sc = flat_press()
    outs = []
    for g in (0, 1):
        ctx = B.Context(sc, precision="mixed", params={"use_graphs": g})
        x, v = dev(sc.X), dev(sc.v_dirichlet)
        for _ in range(2):
            r = ctx.newton_step(x, v)
            assert r["status"] == 0
        outs.append(x.cpu().numpy())
        ctx.close()
    np.testing.assert_array_equal(outs[0], outs[1])
