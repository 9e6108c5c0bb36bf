"""GPU parity of the contact pass (C ABI) against the FP64 CPU oracle.

Tolerances: candidate sets bit-exact; FP64 path relative 1e-12 (energy,
gradient relative L2, Hessian blocks relative Frobenius); mixed path 1e-5 on
energy and gradient and 1e-4 on Hessian blocks; CCD step never larger than
the oracle's (additive CCD bit-identical)."""
import numpy as np
import pytest

from helpers import bsr_dict, hess_blocks_check, hess_rel, rel, small_indent
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
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.12e-3, L=1)
    out.append(("indent_L1", sc, x))
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.12e-3, L=2)
    out.append(("indent_L2", sc, x))
    # three envs of different sizes batched, each pressed differently
    parts, xs = [], []
    for k, (nq, press) in enumerate([(6, 0.08e-3), (9, 0.15e-3), (4, 0.05e-3)]):
        s, xx = small_indent(n_quads=nq, subdiv=2 + (k % 2), press=press, seed=20 + k)
        parts.append(s)
        xs.append(xx)
    out.append(("batch3", S.concat_envs(parts), np.concatenate(xs)))
    return out


SCENES = _scenes()
IDS = [s[0] for s in SCENES]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,sc,x", SCENES, ids=IDS)
def test_candidates_bit_exact(B, oracle_mod, name, sc, x, prec):
    ctx = B.Context(sc, precision=prec)
    O = oracle_mod.Scene(sc)
    for xx in (sc.X, x):
        cnt = ctx.candidates(xx, sc.Y0)
        for kind in range(3):
            g = ctx.candidate_pairs(kind)
            o = O.candidates(kind, xx, sc.Y0)
            np.testing.assert_array_equal(g, o, err_msg=f"kind {kind}")
        assert cnt["face"] == O.candidates(0, xx, sc.Y0).shape[0]
    ctx.close()


@pytest.mark.parametrize("offset", [(37.25, -12.5, 5.125), (-1e3, 2e3, -512.0)])
def test_candidates_far_from_origin(B, oracle_mod, offset):
    """The grid's cell ranges are computed in FP32 with a slack that grows
    with the coordinates' magnitude: a scene far from the origin (cells of
    ~0.1 mm at 40 m and at 2 km) must still give the oracle's exact candidate
    sets, and the swept query the oracle's additive-CCD step."""
    sc, x = small_indent(n_quads=8, subdiv=2, press=0.1e-3, seed=5)
    off = np.asarray(offset)
    import dataclasses
    sc = dataclasses.replace(sc, X=sc.X + off, Y0=sc.Y0 + off)
    x = x + off
    ctx = B.Context(sc, precision="fp64")
    O = oracle_mod.Scene(sc)
    cnt = ctx.candidates(x, sc.Y0)
    for kind in range(3):
        np.testing.assert_array_equal(ctx.candidate_pairs(kind), O.candidates(kind, x, sc.Y0),
                                      err_msg=f"kind {kind}")
    assert cnt["face"] > 0
    dx = np.zeros_like(x)
    dx[:, 2] = -2e-4
    g = ctx.ccd_max_step(x, dx, sc.Y0)
    assert g["alpha_accd"] == O.ccd_max_step(x, dx, sc.Y0)[2]
    assert g["n_pt"] + g["n_ee"] > 0
    ctx.close()


@pytest.mark.parametrize("name,sc,x", SCENES, ids=IDS)
def test_barrier_eval_fp64_parity(B, oracle_mod, name, sc, x):
    ctx = B.Context(sc, precision="fp64")
    O = oracle_mod.Scene(sc)
    r = ctx.barrier_eval(x, sc.Y0)
    o = O.contact(x, sc.Y0)
    assert o["energy"] > 0
    assert r["energy"] == pytest.approx(o["energy"], rel=1e-12)
    assert rel(r["grad"].cpu().numpy(), o["grad"]) < 1e-12
    assert hess_rel(r["hess"], o) < 1e-12
    hess_blocks_check(r["hess"], o, 1e-12)
    c = r["counts"]
    assert (c["point"], c["edge"], c["face"]) == tuple(int(v) for v in o["n_samples"])
    ctx.close()


@pytest.mark.parametrize("name,sc,x", SCENES, ids=IDS)
def test_barrier_eval_mixed_parity(B, oracle_mod, name, sc, x):
    ctx = B.Context(sc, precision="mixed")
    O = oracle_mod.Scene(sc)
    r = ctx.barrier_eval(x, sc.Y0)
    o = O.contact(x, sc.Y0)
    assert r["grad"].dtype == torch.float32
    assert r["energy"] == pytest.approx(o["energy"], rel=1e-5)
    assert rel(r["grad"].cpu().numpy(), o["grad"]) < 1e-5
    assert hess_rel(r["hess"], o) < 1e-4
    hess_blocks_check(r["hess"], o, 1e-4)
    ctx.close()


def test_barrier_eval_deterministic(B):
    sc, x = small_indent(n_quads=12, subdiv=3, press=0.15e-3, L=2)
    for prec in ("fp64", "mixed"):
        ctx = B.Context(sc, precision=prec)
        a = ctx.barrier_eval(x, sc.Y0)
        b = ctx.barrier_eval(x, sc.Y0)
        assert a["energy"] == b["energy"]
        assert torch.equal(a["grad"], b["grad"])
        assert torch.equal(a["hess"][2], b["hess"][2])
        ctx.close()


def test_no_contact_is_zero(B):
    sc, x = small_indent(n_quads=6, subdiv=2)
    ctx = B.Context(sc, precision="fp64")
    r = ctx.barrier_eval(sc.X, sc.Y0)        # rest: 2 dhat away, no contact
    assert r["energy"] == 0.0
    assert float(r["grad"].abs().max()) == 0.0
    assert float(r["hess"][2].abs().max()) == 0.0
    ctx.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ccd_max_step_parity(B, oracle_mod, seed):
    sc, x = small_indent(n_quads=6, subdiv=2, press=0.06e-3, seed=seed)
    ctx = B.Context(sc, precision="fp64")
    O = oracle_mod.Scene(sc)
    rng = np.random.default_rng(seed)
    dx = np.zeros_like(x)
    dx[:, 2] = -(2e-4 + 2e-4 * rng.random(x.shape[0]))
    dx[:, :2] = 3e-5 * rng.normal(size=(x.shape[0], 2))
    g = ctx.ccd_max_step(x, dx, sc.Y0)
    a, al, aa = O.ccd_max_step(x, dx, sc.Y0)
    assert g["alpha_accd"] == aa                      # bit-identical
    assert g["alpha_lin"] <= al and g["alpha_lin"] == pytest.approx(al, rel=1e-9)
    assert g["alpha"] <= a and g["alpha"] == pytest.approx(a, rel=1e-9)
    assert 0 < g["alpha"] < 1
    # the same kind of approach expressed as master motion
    xm1 = sc.Y0 + np.array([0.0, 0.0, 3e-4])
    g2 = ctx.ccd_max_step(x, np.zeros_like(x), sc.Y0, xm1)
    a2, al2, aa2 = O.ccd_max_step(x, np.zeros_like(x), sc.Y0, xm1)
    assert g2["alpha_accd"] == aa2
    assert g2["alpha"] <= a2 and g2["alpha"] == pytest.approx(a2, rel=1e-9)
    ctx.close()


def test_full_size_terrain_sampled_parity(B, oracle_mod):
    """Terrain workload at full size (131,072 slave tris x 16 samples, 199,712
    master tris) in the precision modes the benchmark times: gradient rows and
    Hessian diagonal blocks of sampled contact vertices against the oracle
    evaluated on exactly the slave triangles around them."""
    sc = S.gel_on_terrain()
    x = S.drape_on_master(sc, 0.15e-3)
    O = oracle_mod.Scene(sc)
    for prec, tol_g, tol_h in (("fp64", 1e-12, 1e-12), ("mixed", 1e-5, 1e-4)):
        ctx = B.Context(sc, precision=prec)
        r = ctx.barrier_eval(x, sc.Y0)
        grad = r["grad"].cpu().numpy().astype(np.float64)
        G = bsr_dict(*r["hess"])
        active = np.nonzero(np.abs(grad).sum(axis=1) > 0)[0]
        assert active.shape[0] > 100
        # up to 400 vertices spread over the whole contact front: the active
        # vertices sorted along x, one drawn from each of up to 400 equal strata
        rng = np.random.default_rng(3)
        order = active[np.argsort(x[active, 0], kind="stable")]
        strata = np.array_split(order, min(400, order.shape[0]))
        verts = np.array([s_[rng.integers(len(s_))] for s_ in strata])
        tris = np.unique(np.nonzero(np.isin(sc.stris, verts).any(axis=1))[0])
        o = O.contact(x, sc.Y0, subset=tris)
        # relative L2 over the sampled rows (a single row can be a near-cancelling
        # sum of its triangles' contributions), and every sampled row's blocks
        assert rel(grad[verts], o["grad"][verts]) < tol_g
        hess_blocks_check(r["hess"], o, tol_h, rows=verts)
        ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("moving", [False, True])
def test_contact_pass_fused_matches_separate_and_oracle(B, oracle_mod, prec, moving):
    sc, x = small_indent(n_quads=10, subdiv=3, press=0.1e-3, L=2, seed=4)
    ctx = B.Context(sc, precision=prec)
    O = oracle_mod.Scene(sc)
    rng = np.random.default_rng(9)
    dx = np.zeros_like(x)
    dx[:, 2] = -(1e-5 + 2e-5 * rng.random(x.shape[0]))
    dx[:, :2] = 2e-6 * rng.normal(size=(x.shape[0], 2))
    xm1 = sc.Y0 + np.array([0.0, 0.0, 1e-5]) if moving else None
    r = ctx.contact_pass(x, sc.Y0, dx, xm1)
    e = ctx.barrier_eval(x, sc.Y0)
    c = ctx.ccd_max_step(x, dx, sc.Y0, xm1)
    # same broad phase, same kernels: bitwise equal to the separate calls
    assert r["energy"] == e["energy"]
    assert torch.equal(r["grad"], e["grad"])
    assert torch.equal(r["hess"][2], e["hess"][2])
    assert r["alpha_accd"] == c["alpha_accd"]
    if prec == "fp64" or moving:
        assert (r["alpha"], r["alpha_lin"]) == (c["alpha"], c["alpha_lin"])
    else:
        # mixed, static master: samples evaluated from certified FP32 geometry
        # bound the step with a lower bound of their gap, so the fused pass's
        # alpha_lin never exceeds the FP64 bound of ccd_max_step and stays
        # within 2e-3 of it
        assert r["alpha_lin"] <= c["alpha_lin"] and r["alpha_lin"] >= (1 - 2e-3) * c["alpha_lin"]
        assert r["alpha"] <= c["alpha"] and r["alpha"] >= (1 - 2e-3) * c["alpha"]
    # and against the oracle
    o = O.contact(x, sc.Y0)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert r["energy"] == pytest.approx(o["energy"], rel=tol)
    assert rel(r["grad"].cpu().numpy(), o["grad"]) < tol
    a, al, aa = O.ccd_max_step(x, dx, sc.Y0, xm1)
    arel = 1e-9 if prec == "fp64" or moving else 2e-3
    assert r["alpha_accd"] == aa
    assert r["alpha"] <= a and r["alpha"] == pytest.approx(a, rel=arel)
    if np.isfinite(al):
        assert r["alpha_lin"] <= al and r["alpha_lin"] == pytest.approx(al, rel=arel)
    ctx.close()


def test_mixed_decisions_match_fp64(B):
    """The mixed path makes every sample decision in FP64: the active-sample
    counts equal the FP64 path's on the full-size terrain."""
    sc = S.gel_on_terrain()
    x = S.drape_on_master(sc, 0.15e-3)
    c64 = B.Context(sc, precision="fp64").barrier_eval(x, sc.Y0, hess=False)["counts"]
    c32 = B.Context(sc, precision="mixed").barrier_eval(x, sc.Y0, hess=False)["counts"]
    assert (c32["face"], c32["edge"], c32["point"]) == (c64["face"], c64["edge"], c64["point"])


def test_scattered_surface_inputs_give_the_same_pass(B):
    """ipc_slave_vertices / ipc_scatter_slave: a pass on arrays that hold
    only the slave surface vertices' positions and displacements (the rest
    zero) equals the pass on the full arrays, bitwise."""
    from paper_2605_24339_b300 import scenes as S
    sc = S.gel_on_terrain(n_quads=16, nz=2, terrain_quads=24)
    rng = np.random.default_rng(3)
    x = sc.X.copy()
    x[:, 2] -= 1.5 * sc.params["dhat"]
    dx = rng.normal(scale=1e-5, size=x.shape)
    ctx = B.Context(sc, precision="mixed")
    try:
        xd = torch.as_tensor(x, device="cuda")
        dxd = torch.as_tensor(dx, device="cuda")
        xm = torch.as_tensor(sc.Y0, device="cuda")
        ids = ctx.slave_vertices()
        assert (np.diff(ids) > 0).all() and np.isin(ids, sc.stris.ravel()).all()
        assert len(np.unique(sc.stris)) == len(ids)
        a = ctx.contact_pass(xd, xm, dxd, grad=True, hess=False)
        xs = torch.zeros_like(xd)
        dxs = torch.zeros_like(dxd)
        ctx.scatter_slave(torch.as_tensor(x[ids], device="cuda"), xs)
        ctx.scatter_slave(torch.as_tensor(dx[ids], device="cuda"), dxs)
        b = ctx.contact_pass(xs, xm, dxs, grad=True, hess=False)
        assert a["energy"] == b["energy"] and a["alpha"] == b["alpha"]
        assert torch.equal(a["grad"], b["grad"])
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_host_input_pass_equals_scatter_then_pass(B, prec):
    """ipc_contact_pass_host: the slave vertices' positions and displacements
    copied from page-locked host memory inside the pass (the displacements
    behind the broad phase) give bitwise the pass on the scattered device
    arrays -- energy, gradient, every Hessian block, alpha -- over several
    calls whose host contents change (graph replays read the new values);
    pageable host memory is refused."""
    from paper_2605_24339_b300 import scenes as S
    sc = S.gel_on_terrain(n_quads=16, nz=2, terrain_quads=24)
    rng = np.random.default_rng(5)
    ctx = B.Context(sc, precision=prec)
    try:
        ids = ctx.slave_vertices()
        xm = torch.as_tensor(sc.Y0, device="cuda")
        xs_h = torch.zeros((len(ids), 3), dtype=torch.float64).pin_memory()
        dxs_h = torch.zeros((len(ids), 3), dtype=torch.float64).pin_memory()
        x_a = torch.zeros((sc.X.shape[0], 3), dtype=torch.float64, device="cuda")
        dx_a = torch.zeros_like(x_a)
        x_b, dx_b = torch.zeros_like(x_a), torch.zeros_like(x_a)
        for it in range(4):
            x = sc.X.copy()
            x[:, 2] -= (1.2 + 0.2 * it) * sc.params["dhat"]
            dx = rng.normal(scale=1e-5 * (it + 1), size=x.shape)
            xs_h.copy_(torch.as_tensor(x[ids]))
            dxs_h.copy_(torch.as_tensor(dx[ids]))
            ctx.scatter_slave(torch.as_tensor(x[ids], device="cuda"), x_a)
            ctx.scatter_slave(torch.as_tensor(dx[ids], device="cuda"), dx_a)
            a = ctx.contact_pass(x_a, xm, dx_a, grad=True, hess=True)
            b = ctx.contact_pass_host(xs_h, dxs_h, x_b, dx_b, xm, grad=True, hess=True)
            assert torch.equal(x_a, x_b) and torch.equal(dx_a, dx_b)
            assert a["energy"] == b["energy"] and a["alpha"] == b["alpha"], it
            assert a["alpha_lin"] == b["alpha_lin"] and a["alpha_accd"] == b["alpha_accd"]
            assert torch.equal(a["grad"], b["grad"])
            for pa, pb in zip(a["hess"], b["hess"]):   # row_ptr, col_idx, blocks
                assert torch.equal(pa, pb)
        with pytest.raises(B.GmcpError):
            ctx.contact_pass_host(torch.zeros((len(ids), 3), dtype=torch.float64), None, x_b, None, xm)
    finally:
        ctx.close()
