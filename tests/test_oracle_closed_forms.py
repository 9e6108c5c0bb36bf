"""Hand-worked closed forms for each sample kind of the oracle's potential.

Each scene has one slave triangle and a master built so that the active
samples, their weights, their smoothing factors gamma and their gaps follow
from plane geometry by hand (the derivations are in ``tests/golden/``):

* a point sample (Sec. 4.1 "Point samples": weight 1, gamma 1);
* two edge samples of an edge clipped near its start (Sec. 4.1 "Edge samples",
  Sec. 4.3 Eq. gamma: both Gauss points inside the delta_e band, so gamma,
  the Gauss points and the weight ell/2 all enter);
* face samples with one centroid outside the master, one inside the delta_T
  band and one clear of it (Sec. 4.1 "Face samples", Sec. 4.3 Eq. gamma),
  together with the edge samples of the master edge that crosses the slave.

A dropped smoothing factor, a wrong Gauss point, a doubled weight or a wrong
point weight each changes Psi by a factor far outside the 1e-12 tolerance.
"""
import numpy as np
import pytest

from helpers import MM, edge_master, face_master, load_golden, one_slave_triangle, spike_master

Z = np.array([0.0, 0.0, 1.0])


def B(g, eps):
    """IPC barrier and its derivative (Sec. 4.2), written out here so that the
    expectation does not come from the oracle."""
    d = g - eps
    L = np.log(g / eps)
    return -d * d * L, -2.0 * d * L - d * d / g


def _slave_grad(x_mm, y_mm, c1):
    """Gradient rows of the three slave vertices for one sample at (x, y) mm of
    the slave triangle with coefficient c1 = kappa w gamma B'(g):
    grad_a = -c1 beta^s_a n_s = c1 beta^s_a (0, 0, 1)."""
    bs = np.array([1.0 - x_mm - y_mm, y_mm, x_mm])
    return c1 * bs[:, None] * Z[None, :]


@pytest.mark.parametrize("row", list(load_golden("closed_form_point_sample.txt")))
def test_point_sample_closed_form(oracle_mod, row):
    g, w, gamma, bs = row[0], row[1], row[2], row[3:6]
    Y, F = spike_master((0.3, 0.2), g)
    sc, x, xm = one_slave_triangle(Y, F)
    O = oracle_mod.Scene(sc)
    kp, dhat = sc.params["kappa_point"], sc.params["dhat"]
    smp = O.samples(x, xm)
    assert smp.shape[0] == 1 and smp[0, 0] == 0
    assert smp[0, 3] == pytest.approx(g, rel=1e-12)
    assert smp[0, 4] == dhat
    assert smp[0, 5] == w and smp[0, 6] == gamma and smp[0, 7] == kp
    np.testing.assert_allclose(smp[0, 8:11], bs, rtol=0, atol=1e-15)
    r = O.contact(x, xm)
    Bv, dB = B(g, dhat)
    assert r["energy"] == pytest.approx(kp * w * gamma * Bv, rel=1e-12)
    exp = np.zeros_like(x)
    exp[:3] = kp * w * gamma * dB * bs[:, None] * Z[None, :]
    np.testing.assert_allclose(r["grad"], exp, rtol=0, atol=1e-12 * np.abs(exp).max())


@pytest.mark.parametrize("row", list(load_golden("closed_form_edge_sample.txt")))
def test_edge_samples_closed_form(oracle_mod, row):
    gA, gB = row[0], row[1]
    eta, gamma, w = row[2:4], row[4:6], row[6]
    Y, F = edge_master(gA, gB)
    sc, x, xm = one_slave_triangle(Y, F)
    O = oracle_mod.Scene(sc)
    ke, dhat = sc.params["kappa_edge"], sc.params["dhat"]
    gq = gA + eta * (gB - gA)
    xq = -0.01 + 10.0 * eta                    # mm, on y = 0.25 mm
    smp = O.samples(x, xm)
    assert smp.shape[0] == 2 and np.all(smp[:, 0] == 1)
    smp = smp[np.argsort(smp[:, 10])]          # by beta^s_2 = x
    np.testing.assert_allclose(smp[:, 3], gq, rtol=1e-12)
    np.testing.assert_allclose(smp[:, 5], [w, w], rtol=1e-12)
    np.testing.assert_allclose(smp[:, 6], gamma, rtol=1e-12)
    np.testing.assert_allclose(smp[:, 10], xq, rtol=1e-12)
    r = O.contact(x, xm)
    E = 0.0
    G = np.zeros_like(x)
    for q in range(2):
        Bv, dB = B(gq[q], dhat)
        E += ke * w * gamma[q] * Bv
        G[:3] += _slave_grad(xq[q], 0.25, ke * w * gamma[q] * dB)
    assert r["energy"] == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(r["grad"], G, rtol=0, atol=1e-12 * np.abs(G).max())


def _face_gamma_rows():
    return load_golden("closed_form_face_gamma.txt")


@pytest.mark.parametrize("g", [1e-5, 3e-5, 8e-5])
@pytest.mark.parametrize("with_edges", [False, True], ids=["face_only", "face_and_edge"])
def test_face_gamma_closed_form(oracle_mod, g, with_edges):
    rows = _face_gamma_rows()
    Y, F = face_master(g)
    sc, x, xm = one_slave_triangle(Y, F, kappa_edge=1e2 if with_edges else 0.0,
                                   kappa_point=1e-1 if with_edges else 0.0)
    O = oracle_mod.Scene(sc)
    k, ke, dhat = sc.params["kappa"], sc.params["kappa_edge"], sc.params["dhat"]
    A = 0.5 * MM * MM
    Bv, dB = B(g, dhat)
    inside = rows[rows[:, 3] >= 0]
    smp = O.samples(x, xm)
    face = smp[smp[:, 0] == 2]
    assert face.shape[0] == inside.shape[0]
    # match each face sample to its centroid by beta^s = (1-x-y, y, x)
    for rrow in inside:
        hit = face[(np.abs(face[:, 10] - rrow[0]) < 1e-12) & (np.abs(face[:, 9] - rrow[1]) < 1e-12)]
        assert hit.shape[0] == 1
        assert hit[0, 5] == pytest.approx(A / 4, rel=1e-12)
        assert hit[0, 6] == pytest.approx(rrow[3], rel=1e-12)
    E = k * (A / 4) * inside[:, 3].sum() * Bv
    G = np.zeros_like(x)
    for rrow in inside:
        G[:3] += _slave_grad(rrow[0], rrow[1], k * (A / 4) * rrow[3] * dB)
    edge = smp[smp[:, 0] == 1]
    assert edge.shape[0] == 2                  # counted even when kappa_edge = 0
    assert np.all(smp[:, 0] != 0)
    np.testing.assert_allclose(edge[:, 5], [0.41 * MM, 0.41 * MM], rtol=1e-12)
    np.testing.assert_allclose(edge[:, 6], [1.0, 1.0], rtol=0)
    E += ke * 0.82 * MM * Bv
    yq = 0.41 + np.array([-1.0, 1.0]) * 0.41 / np.sqrt(3.0)
    for q in range(2):
        G[:3] += _slave_grad(0.18, yq[q], ke * 0.41 * MM * dB)
    r = O.contact(x, xm)
    assert r["energy"] == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(r["grad"], G, rtol=0, atol=1e-12 * np.abs(G).max())


def test_face_gamma_band_matters(oracle_mod):
    """The smoothing factor of the band sample is what separates the two
    expectations: with gamma = 1 everywhere the face part would be 2/1.733 of
    the hand value."""
    rows = _face_gamma_rows()
    inside = rows[rows[:, 3] >= 0]
    assert 0.0 < inside[:, 3].min() < 1.0
    assert inside[:, 2].min() < 0.1 < inside[:, 2].max()


@pytest.mark.parametrize("kind", ["point", "edge"])
def test_support_radius_from_rest_gap(oracle_mod, kind):
    """Sec. 4.4 Eq. (adaptive_eps) with reading R5: a sample whose rest gap
    g_ref is below dhat/0.9 takes eps = 0.9 g_ref.  The rest master here is
    2e-5 m lower than the current one, so g_ref = g + 2e-5 per sample."""
    lift = 2e-5
    if kind == "point":
        Y, F = spike_master((0.3, 0.2), 3e-5)
        gq = np.array([3e-5])
    else:
        Y, F = edge_master(2e-5, 4e-4)
        eta = load_golden("closed_form_edge_sample.txt")[1, 2:4]
        gq = 2e-5 + eta * (4e-4 - 2e-5)
    sc, x, xm = one_slave_triangle(Y, F, gap_rest=lift)
    O = oracle_mod.Scene(sc)
    smp = O.samples(x, xm)
    smp = smp[np.argsort(smp[:, 3])]
    np.testing.assert_allclose(smp[:, 3], gq, rtol=1e-12)
    np.testing.assert_allclose(smp[:, 4], 0.9 * (gq + lift), rtol=1e-12)
    assert np.all(smp[:, 4] < sc.params["dhat"])
