"""GPU master rows (ipc_master_grad through the C ABI) against the oracle's
(Sec. 4.3 with Eq. gap).  Both evaluate the samples in FP64 and sum in
different orders, so the comparison is relative 1e-11 of the largest row;
the GPU sums each row in a fixed order (entries sorted by master vertex,
then by value), so repeated calls agree bitwise."""
import numpy as np
import pytest

from helpers import flat_over_big_triangle, small_indent
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


def _scenes():
    out = []
    for L in (1, 2):
        sc, x = small_indent(n_quads=10, subdiv=3, press=0.12e-3, L=L)
        out.append((f"indent_L{L}", sc, x))
    parts, xs = [], []
    for k, (nq, press) in enumerate([(6, 0.08e-3), (9, 0.15e-3), (4, 0.05e-3)]):
        s, xx = small_indent(n_quads=nq, subdiv=2 + (k % 2), press=press, seed=20 + k)
        parts.append(s)
        xs.append(xx)
    out.append(("batch3", S.concat_envs(parts), np.concatenate(xs)))
    return out


SCENES = _scenes()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,sc,x", SCENES, ids=[s[0] for s in SCENES])
def test_master_grad_matches_oracle(B, oracle_mod, name, sc, x, prec):
    ctx = B.Context(sc, precision=prec)
    O = oracle_mod.Scene(sc)
    g = ctx.master_grad(x, sc.Y0).cpu().numpy()
    o = O.master_grad(x, sc.Y0)
    scale = np.abs(o).max()
    assert scale > 0
    np.testing.assert_allclose(g, o, rtol=0, atol=1e-11 * scale)
    # rows only where the oracle has them
    assert np.array_equal(np.any(g != 0, axis=1), np.any(o != 0, axis=1))
    # balance with the slave rows of the same pass (FP64 context)
    if prec == "fp64":
        gs = ctx.barrier_eval(x, sc.Y0, hess=False, counts=False)["grad"].cpu().numpy()
        np.testing.assert_allclose(g.sum(axis=0), -gs.sum(axis=0), rtol=0, atol=1e-11 * np.abs(gs).sum())
    ctx.close()


def test_master_grad_no_contact_and_repeat(B):
    sc, x, xm = flat_over_big_triangle(nq=2, gap=2e-4)
    ctx = B.Context(sc, precision="fp64")
    assert np.all(ctx.master_grad(x, xm).cpu().numpy() == 0.0)
    sc2, x2 = small_indent(n_quads=8, subdiv=2, press=0.12e-3)
    ctx2 = B.Context(sc2, precision="fp64")
    a = ctx2.master_grad(x2, sc2.Y0).cpu().numpy()
    b = ctx2.master_grad(x2, sc2.Y0).cpu().numpy()
    assert np.abs(a).max() > 0
    np.testing.assert_array_equal(a.view(np.int64), b.view(np.int64))   # fixed-order sums
    ctx.close()
    ctx2.close()


def test_full_size_terrain_sampled_master_rows(B, oracle_mod):
    """gel_on_terrain at full size (131,072 slave tris x 16 samples, 199,712
    master tris) in the mixed mode the benchmark times: sampled master rows
    against the oracle evaluated on every slave triangle near the sampled
    vertices (a superset of the triangles that can reach them), and the
    force balance with the slave rows over the whole pass."""
    sc = S.gel_on_terrain()
    x = S.drape_on_master(sc, 0.15e-3)
    ctx = B.Context(sc, precision="mixed")
    g = ctx.master_grad(x, sc.Y0).cpu().numpy()
    assert np.any(g != 0, axis=1).sum() > 100
    Y, M, T = sc.Y0, sc.mtris, sc.stris
    lm = np.linalg.norm(Y[M] - Y[M[:, [1, 2, 0]]], axis=2).max()
    ls = np.linalg.norm(x[T] - x[T[:, [1, 2, 0]]], axis=2).max()
    radius = 2.0 * (lm + ls) + sc.params["dhat"]
    cen = x[T].mean(axis=1)
    from scipy.spatial import cKDTree
    tree = cKDTree(cen)
    # master vertices closer than half a slave edge to a slave centroid
    # (geometry only: most of them carry contact)
    near = np.flatnonzero(tree.query(Y)[0] < 0.5 * ls)
    rng = np.random.default_rng(3)
    O = oracle_mod.Scene(sc)
    n_nonzero = 0
    for u in rng.choice(near, 12, replace=False):
        sub = np.array(sorted(tree.query_ball_point(Y[u], radius)), dtype=np.int32)
        o = O.master_grad(x, sc.Y0, subset=sub)
        np.testing.assert_allclose(g[u], o[u], rtol=0, atol=1e-11 * max(np.abs(o[u]).max(), 1e-300))
        n_nonzero += bool(np.any(o[u] != 0))
    assert n_nonzero >= 5
    ctx64 = B.Context(sc, precision="fp64")
    gs = ctx64.barrier_eval(x, sc.Y0, hess=False, counts=False)["grad"].cpu().numpy()
    np.testing.assert_allclose(g.sum(axis=0), -gs.sum(axis=0), rtol=0, atol=1e-11 * np.abs(gs).sum())
    ctx.close()
    ctx64.close()


def _sum_blocks(ij, blk):
    out = {}
    for (r, c), b in zip(ij.cpu().numpy(), blk.cpu().numpy()):
        key = (int(r), int(c))
        out[key] = out.get(key, 0.0) + b
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,sc,x", SCENES, ids=[s[0] for s in SCENES])
def test_master_hess_matches_oracle(B, oracle_mod, name, sc, x, prec):
    ctx = B.Context(sc, precision=prec)
    O = oracle_mod.Scene(sc)
    G = _sum_blocks(*ctx.master_hess(x, sc.Y0, capacity=16))   # grows once
    H = O.master_hess(x, sc.Y0)
    assert set(G) == set(H)
    scale = max(np.abs(b).max() for b in H.values())
    for k, b in H.items():
        np.testing.assert_allclose(G[k], b, rtol=0, atol=1e-11 * scale)
    ctx.close()


def test_master_hess_capacity_and_empty(B):
    sc, x = small_indent(n_quads=8, subdiv=2, press=0.12e-3)
    ctx = B.Context(sc, precision="fp64")
    ij, blk = ctx.master_hess(x, sc.Y0)
    n = ij.shape[0]
    assert n > 0
    # too small: IPC_ERR_CAPACITY with the count, nothing past capacity written
    import ctypes
    from paper_2605_24339_b300 import binding as Bm
    xs, xm = ctx._as(x), ctx._as(sc.Y0)
    ij2 = torch.full((4, 2), -7, dtype=torch.int32, device="cuda")
    blk2 = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
    cnt = ctypes.c_int64()
    st = Bm.lib().ipc_master_hess(ctx.h, Bm._ptr(xs), Bm._ptr(xm), 2, Bm._ptr(ij2), Bm._ptr(blk2), ctypes.byref(cnt))
    assert st == 5 and cnt.value == n
    assert (ij2[2:].cpu().numpy() == -7).all()
    # argument errors are statuses, not faults
    st = Bm.lib().ipc_master_hess(ctx.h, Bm._ptr(xs), Bm._ptr(xm), -1, Bm._ptr(ij2), Bm._ptr(blk2), ctypes.byref(cnt))
    assert st == 1
    st = Bm.lib().ipc_master_hess(ctx.h, Bm._ptr(xs), None, 4, Bm._ptr(ij2), Bm._ptr(blk2), ctypes.byref(cnt))
    assert st == 1
    st = Bm.lib().ipc_master_grad(ctx.h, Bm._ptr(xs), Bm._ptr(xm), None)
    assert st == 1
    # no contact: no blocks
    sc3, x3, xm3 = flat_over_big_triangle(nq=2, gap=2e-4)
    ctx3 = B.Context(sc3, precision="fp64")
    ij3, _ = ctx3.master_hess(x3, xm3)
    assert ij3.shape[0] == 0
    ctx.close()
    ctx3.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_warp_per_triangle_path_gives_the_same_results(B, oracle_mod, prec):
    """An item buffer too small for the items sends the evaluation and both
    master modes to the warp-per-triangle kernel: the same results as the
    item-parallel kernels, and the oracle's."""
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.12e-3, L=2)
    O = oracle_mod.Scene(sc)
    a = B.Context(sc, precision=prec)
    b = B.Context(sc, precision=prec)
    b.set_item_capacity(1)
    ra = a.barrier_eval(x, sc.Y0, hess=False)
    rb = b.barrier_eval(x, sc.Y0, hess=False)
    assert all(rb["counts"][k] == ra["counts"][k] for k in ("face", "edge", "point"))
    ga, gb = ra["grad"].cpu().numpy(), rb["grad"].cpu().numpy()
    if prec == "fp64":
        np.testing.assert_array_equal(gb, ga)     # same sums in the same order
    else:
        np.testing.assert_allclose(gb, ga, rtol=0, atol=1e-6 * np.abs(ga).max())
    o = O.master_grad(x, sc.Y0)
    for ctx in (a, b):
        np.testing.assert_allclose(ctx.master_grad(x, sc.Y0).cpu().numpy(), o, rtol=0,
                                   atol=1e-11 * np.abs(o).max())
    H = O.master_hess(x, sc.Y0)
    G = _sum_blocks(*b.master_hess(x, sc.Y0))
    assert set(G) == set(H)
    scale = max(np.abs(v).max() for v in H.values())
    for k, v in H.items():
        np.testing.assert_allclose(G[k], v, rtol=0, atol=1e-11 * scale)
    with pytest.raises(B.GmcpError):
        b.set_item_capacity(0)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_master_rows_with_a_deformed_master(B, oracle_mod, prec):
    """The master away from its rest shape (rest gaps and eps from Y0, the
    geometry from the current master): rows and blocks as the oracle's."""
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.10e-3, L=1)
    rng = np.random.default_rng(5)
    Y = sc.Y0
    c = Y.mean(axis=0)
    xm = c + (Y - c) * np.array([1.01, 0.99, 1.0]) + rng.normal(scale=2e-6, size=Y.shape)
    xm[:, 2] += 0.02e-3
    O = oracle_mod.Scene(sc)
    o = O.master_grad(x, xm)
    assert np.abs(o).max() > 0
    ctx = B.Context(sc, precision=prec)
    np.testing.assert_allclose(ctx.master_grad(x, xm).cpu().numpy(), o, rtol=0, atol=1e-11 * np.abs(o).max())
    H = O.master_hess(x, xm)
    G = _sum_blocks(*ctx.master_hess(x, xm))
    assert set(G) == set(H)
    scale = max(np.abs(v).max() for v in H.values())
    for k, v in H.items():
        np.testing.assert_allclose(G[k], v, rtol=0, atol=1e-11 * scale)
    ctx.close()
