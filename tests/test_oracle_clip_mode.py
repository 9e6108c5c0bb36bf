"""Pins of the oracle's contact potential with the paper's clipped-overlap
face samples (Sec. 4.1 "Face samples", face_sampler = 1): closed forms where
the overlap area is known by hand, and the derivative and PSD invariants of
the fixed-rule mode.

* Full cover: a flat pad over one large facing master triangle: each slave
  triangle's clipped overlap is itself, one fan triangle with three Gauss
  samples of weight A/3, so Psi = kappa A_pad B(g).
* Partial overlap: the one-triangle scene of tests/golden/closed_form_face_
  gamma.txt: the master M0=(0.18,-1), M1=(2.5,-1), M2=(0.18,2.5) mm covers the
  part x >= 0.18 mm of the slave triangle (0,0),(0,1),(1,0) mm, the triangle
  (0.18,0), (1,0), (0.18,0.82) mm of area 0.82^2/2 mm^2.  With delta_T
  shrunk to 1e-9 every Gauss point is clear of the smoothing band, so the
  face part is kappa 0.3362e-6 B(g) whatever fan the clipper forms.
"""
import numpy as np
import pytest

from helpers import MM, face_master, flat_over_big_triangle, one_slave_triangle, small_indent


def B(g, eps):
    d = g - eps
    return -d * d * np.log(g / eps)


@pytest.mark.parametrize("g", [1e-5, 4e-5, 8e-5])
def test_full_cover_closed_form(oracle_mod, g):
    sc, x, xm = flat_over_big_triangle(nq=3, gap=g, L=1)
    sc.params["face_sampler"] = 1
    O = oracle_mod.Scene(sc)
    r = O.contact(x, xm)
    A = (3e-3) ** 2
    assert r["n_samples"][2] == 3 * sc.stris.shape[0]
    assert r["energy"] == pytest.approx(sc.params["kappa"] * A * B(g, sc.params["dhat"]), rel=1e-12)
    smp = O.samples(x, xm)
    areas = 0.5 * np.linalg.norm(np.cross(x[sc.stris[:, 1]] - x[sc.stris[:, 0]],
                                          x[sc.stris[:, 2]] - x[sc.stris[:, 0]]), axis=1)
    for t in range(sc.stris.shape[0]):
        w = smp[smp[:, 1] == t, 5]
        np.testing.assert_allclose(w, areas[t] / 3, rtol=1e-12)


@pytest.mark.parametrize("g", [1e-5, 3e-5, 8e-5])
def test_partial_overlap_closed_form(oracle_mod, g):
    Y, F = face_master(g)
    sc, x, xm = one_slave_triangle(Y, F, kappa_edge=0.0, kappa_point=0.0)
    sc.params.update(face_sampler=1, delta_T=1e-9)
    O = oracle_mod.Scene(sc)
    smp = O.samples(x, xm)
    face = smp[smp[:, 0] == 2]
    assert face.shape[0] >= 3 and face.shape[0] % 3 == 0
    A_ov = 0.5 * 0.82 ** 2 * MM * MM
    assert face[:, 5].sum() == pytest.approx(A_ov, rel=1e-12)
    assert np.all(face[:, 6] == 1.0)
    r = O.contact(x, xm)
    assert r["energy"] == pytest.approx(sc.params["kappa"] * A_ov * B(g, sc.params["dhat"]), rel=1e-12)
    # every Gauss point lies in the overlap: x >= 0.18 mm (beta^s_2 = x / 1 mm)
    assert np.all(face[:, 10] >= 0.18 - 1e-12)


def _dense_hessian(nv, blk_ij, blk):
    H = np.zeros((3 * nv, 3 * nv))
    for (i, j), b in zip(blk_ij, blk):
        H[3 * i:3 * i + 3, 3 * j:3 * j + 3] += b
    return H


def test_clip_mode_lagged_fd_and_psd(oracle_mod):
    """Reading R6 holds in clip mode too: the gradient and Hessian are the
    exact derivatives of the frozen-linear potential, every block is PSD."""
    sc, x = small_indent(L=1)
    sc.params["face_sampler"] = 1
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    assert r["n_samples"][2] > 30
    H = _dense_hessian(sc.X.shape[0], r["blk_ij"], r["blk"])
    rng = np.random.default_rng(0)
    for _ in range(2):
        d = rng.normal(size=x.shape) * 1e-6
        h = 1e-3
        E = O.lagged(x, sc.Y0, d, [-h, 0.0, h])
        assert E[1] == pytest.approx(r["energy"], rel=1e-14)
        assert (E[2] - E[0]) / (2 * h) == pytest.approx(np.sum(r["grad"] * d), rel=1e-6)
        assert (E[2] - 2 * E[1] + E[0]) / h ** 2 == pytest.approx(d.ravel() @ H @ d.ravel(), rel=1e-4)
    for b in r["blk"]:
        w = np.linalg.eigvalsh(0.5 * (b + b.T))
        assert w.min() >= -1e-12 * max(abs(w).max(), 1e-300)


def test_clip_mode_rest_state_and_broad_phase(oracle_mod):
    """The rest state carries no force (Eq. adaptive_eps with the rest gap of
    each clipped sample's slave point); the box-box face candidates are
    conservative: all pairs give the same samples bit for bit."""
    sc, x, xm = flat_over_big_triangle(nq=2, gap=5e-5, rest_gap=5e-5, face_only=False)
    sc.params["face_sampler"] = 1
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    assert r["energy"] == 0.0 and np.all(r["grad"] == 0.0)
    sc2, x2 = small_indent(L=1)
    sc2.params["face_sampler"] = 1
    O2 = oracle_mod.Scene(sc2)
    a = O2.contact(x2, sc2.Y0)
    O2.set_all_pairs(True)
    b = O2.contact(x2, sc2.Y0)
    assert a["energy"] == b["energy"]
    np.testing.assert_array_equal(a["grad"], b["grad"])
