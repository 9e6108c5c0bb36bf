"""The GPU contact pass on the hand-worked scenes whose potential has a
closed form (derivations in tests/golden/closed_form_*.txt): a point sample
(Sec. 4.1 "Point samples"), two edge samples inside the delta_e band of
their edge (Sec. 4.1 "Edge samples", Sec. 4.3 Eq. gamma) and face samples
with one inside the delta_T band beside a crossing master edge.  Energy and
gradient against the closed form and the oracle: 1e-12 (FP64 path), 1e-5
(mixed); Hessian blocks per block: 1e-12 / 1e-4; candidate sets bit-exact."""
import numpy as np
import pytest

from helpers import (MM, edge_master, face_master, hess_blocks_check, load_golden, one_slave_triangle, rel,
                     spike_master)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24339_b300 import binding
    binding.lib()
    return binding


def Bv(g, eps):
    d = g - eps
    return -d * d * np.log(g / eps)


def _cases():
    out = []
    for g in load_golden("closed_form_point_sample.txt")[:, 0]:
        Y, F = spike_master((0.3, 0.2), g)
        out.append((f"point_g{g:.0e}", Y, F, {}, None))
    for row in load_golden("closed_form_edge_sample.txt"):
        gA, gB, eta, gam, w = row[0], row[1], row[2:4], row[4:6], row[6]
        Y, F = edge_master(gA, gB)
        gq = gA + eta * (gB - gA)
        out.append((f"edge_{gA:.0e}_{gB:.0e}", Y, F, {}, ("edge", gq, gam, w)))
    fr = load_golden("closed_form_face_gamma.txt")
    gsum = fr[fr[:, 3] >= 0, 3].sum()
    for g in (1e-5, 3e-5, 8e-5):
        Y, F = face_master(g)
        out.append((f"face_g{g:.0e}", Y, F, {}, ("face", g, gsum)))
    return out


CASES = _cases()


def _expected(sc, Y, extra):
    p = sc.params
    dh = p["dhat"]
    if extra is None:                       # point: apex depth is the gap
        return p["kappa_point"] * Bv(-Y[0, 2], dh)
    if extra[0] == "edge":
        _, gq, gam, w = extra
        return sum(p["kappa_edge"] * w * gam[q] * Bv(gq[q], dh) for q in range(2))
    _, g, gsum = extra
    return (p["kappa"] * 0.125 * MM * MM * gsum + p["kappa_edge"] * 0.82 * MM) * Bv(g, dh)


@pytest.mark.parametrize("prec,tol,tol_h", [("fp64", 1e-12, 1e-12), ("mixed", 1e-5, 1e-4)])
@pytest.mark.parametrize("name,Y,F,kw,extra", CASES, ids=[c[0] for c in CASES])
def test_closed_form_scene(B, oracle_mod, name, Y, F, kw, extra, prec, tol, tol_h):
    sc, x, xm = one_slave_triangle(Y, F, **kw)
    ctx = B.Context(sc, precision=prec)
    O = oracle_mod.Scene(sc)
    try:
        r = ctx.barrier_eval(x, xm)
        o = O.contact(x, xm)
        E = _expected(sc, Y, extra)
        assert o["energy"] == pytest.approx(E, rel=1e-12)
        assert r["energy"] == pytest.approx(E, rel=tol)
        assert rel(r["grad"].cpu().numpy(), o["grad"]) < tol
        hess_blocks_check(r["hess"], o, tol_h)
        c = r["counts"]
        assert (c["point"], c["edge"], c["face"]) == tuple(int(v) for v in o["n_samples"])
        for kind in range(3):
            np.testing.assert_array_equal(ctx.candidate_pairs(kind), O.candidates(kind, x, xm))
    finally:
        ctx.close()
