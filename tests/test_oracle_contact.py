"""Pins of the oracle's contact potential (Sec. 4.1-4.5) against closed forms,
invariants and finite differences."""
import numpy as np
import pytest

from helpers import flat_over_big_triangle, rotation, small_indent


def test_flat_closed_form_energy(oracle_mod):
    # A flat pad at uniform gap g over one facing master triangle, far from
    # its edges (gamma = 1), face samples only, eps = eps_max (rest gap large):
    # Psi = kappa * A_pad * B(g, eps) exactly (weights sum to the area).
    for L in (1, 2):
        for g in (1e-5, 3e-5, 8e-5):
            sc, x, xm = flat_over_big_triangle(nq=3, gap=g, L=L)
            O = oracle_mod.Scene(sc)
            r = O.contact(x, xm)
            B, dB, _ = oracle_mod.barrier(g, sc.params["dhat"])
            A = (3e-3) ** 2
            kappa = sc.params["kappa"]
            assert r["energy"] == pytest.approx(kappa * A * B, rel=1e-12)
            assert r["n_samples"][2] == 2 * 9 * 4 ** L
            # total gradient = -kappa A B'(g) n_s, n_s = -z
            tot = r["grad"].sum(axis=0)
            np.testing.assert_allclose(tot, [0, 0, kappa * A * dB], rtol=1e-12, atol=1e-30)


def test_flat_normal_translation_fd(oracle_mod):
    # For parallel planes the paper's gradient is the exact derivative of the
    # true Psi along a rigid normal translation of the pad.
    sc, x, xm = flat_over_big_triangle(nq=2, gap=4e-5, face_only=False)
    O = oracle_mod.Scene(sc)
    r = O.contact(x, xm)
    d = np.zeros_like(x)
    d[:, 2] = -1.0
    h = 1e-10
    xp, xmn = x + h * d, x - h * d
    fd = (O.contact(xp, xm)["energy"] - O.contact(xmn, xm)["energy"]) / (2 * h)
    assert fd == pytest.approx(np.sum(r["grad"] * d), rel=1e-6)


def test_rest_state_has_no_force(oracle_mod):
    # Sec. 4.4: with eps = min(0.9 g_ref, eps_max) the rest configuration
    # carries no barrier energy or force even when the master is within eps_max.
    sc, x, xm = flat_over_big_triangle(nq=2, gap=5e-5, rest_gap=5e-5, face_only=False)
    O = oracle_mod.Scene(sc)
    assert O.candidates(0, x, xm).shape[0] > 0
    r = O.contact(x, sc.Y0)
    assert r["energy"] == 0.0
    assert np.all(r["grad"] == 0.0)
    sc2, x2 = small_indent()
    sc2.Y0[:, 2] += 1.5e-4      # apex now 0.5 dhat below the rest pad
    O2 = oracle_mod.Scene(sc2)
    assert O2.candidates(0, sc2.X, sc2.Y0).shape[0] > 0
    r2 = O2.contact(sc2.X, sc2.Y0)
    assert r2["energy"] == 0.0 and np.all(r2["grad"] == 0.0)
    # pressing further (rigidly, by 0.2 of that gap) creates energy
    x3 = sc2.X.copy()
    x3[:, 2] -= 0.1e-4
    assert O2.contact(x3, sc2.Y0)["energy"] > 0.0


def test_rigid_invariance(oracle_mod):
    sc, x = small_indent()
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    assert r["energy"] > 0
    R = rotation(3)
    T = np.array([0.3, -0.2, 0.1])
    sc.X = sc.X @ R.T + T
    sc.Y0 = sc.Y0 @ R.T + T
    O2 = oracle_mod.Scene(sc)
    r2 = O2.contact(x @ R.T + T, sc.Y0)
    assert r2["energy"] == pytest.approx(r["energy"], rel=1e-8)
    np.testing.assert_array_equal(r2["n_samples"], r["n_samples"])
    np.testing.assert_allclose(r2["grad"], r["grad"] @ R.T, rtol=0,
                               atol=1e-7 * np.abs(r["grad"]).max())


def _dense_hessian(nv, blk_ij, blk):
    H = np.zeros((3 * nv, 3 * nv))
    for (i, j), b in zip(blk_ij, blk):
        H[3 * i:3 * i + 3, 3 * j:3 * j + 3] += b
    return H


def test_lagged_potential_fd(oracle_mod):
    # Reading R6: the paper's gradient and Hessian are the exact derivatives
    # of the frozen-linear potential of the current samples.
    sc, x = small_indent(L=2)
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    assert r["n_samples"].sum() > 50
    rng = np.random.default_rng(0)
    H = _dense_hessian(sc.X.shape[0], r["blk_ij"], r["blk"])
    for trial in range(3):
        d = rng.normal(size=x.shape) * 1e-6
        h = 1e-3
        E = O.lagged(x, sc.Y0, d, [-h, 0.0, h])
        assert E[1] == pytest.approx(r["energy"], rel=1e-14)
        gd = np.sum(r["grad"] * d)
        assert (E[2] - E[0]) / (2 * h) == pytest.approx(gd, rel=1e-6)
        dHd = d.ravel() @ H @ d.ravel()
        assert (E[2] - 2 * E[1] + E[0]) / h ** 2 == pytest.approx(dHd, rel=1e-4)


def test_hessian_psd(oracle_mod):
    sc, x = small_indent()
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    for b in r["blk"]:
        w = np.linalg.eigvalsh(0.5 * (b + b.T))
        assert w.min() >= -1e-12 * max(abs(w).max(), 1e-300)
    H = _dense_hessian(sc.X.shape[0], r["blk_ij"], r["blk"])
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    w = np.linalg.eigvalsh(H)
    assert w.min() >= -1e-10 * w.max()


def test_broad_phase_is_conservative(oracle_mod):
    # every pair that carries an active sample is a candidate: testing all
    # pairs gives the same samples and the same energy bit for bit
    sc, x = small_indent()
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    O.set_all_pairs(True)
    r2 = O.contact(x, sc.Y0)
    assert r2["energy"] == r["energy"]
    np.testing.assert_array_equal(r2["grad"], r["grad"])


def test_candidate_predicates_by_hand(oracle_mod):
    # face pairs: some face sample inside the master tri box grown by dhat
    sc, x = small_indent()
    O = oracle_mod.Scene(sc)
    xm = sc.Y0
    dh = sc.params["dhat"]
    rule = oracle_mod.face_rule(1)
    cand = {tuple(p) for p in O.candidates(0, x, xm)}
    rng = np.random.default_rng(1)
    sel_s = rng.choice(sc.stris.shape[0], 40, replace=False)
    for s in sel_s:
        samp = rule @ x[sc.stris[s]]
        for m in range(sc.mtris.shape[0]):
            lo = xm[sc.mtris[m]].min(axis=0) - dh
            hi = xm[sc.mtris[m]].max(axis=0) + dh
            inside = np.any(np.all((samp >= lo) & (samp <= hi), axis=1))
            assert inside == ((s, m) in cand)
    # point pairs: master vertex box vs slave tri box
    cand = {tuple(p) for p in O.candidates(2, x, xm)}
    for s in sel_s:
        lo, hi = x[sc.stris[s]].min(axis=0), x[sc.stris[s]].max(axis=0)
        hit = np.all((lo <= xm + dh) & (xm - dh <= hi), axis=1)
        got = {m for (t, m) in cand if t == s}
        assert got == set(np.nonzero(hit)[0].tolist())


def test_linearised_step_hits_tenth_of_gap(oracle_mod):
    # Eq. (ccd): at alpha_lin the critical linearised gap is 0.1 g_k, so the
    # frozen-linear gap reaches zero exactly at alpha_lin / 0.9.
    sc, x = small_indent()
    O = oracle_mod.Scene(sc)
    rng = np.random.default_rng(2)
    d = np.zeros_like(x)
    d[:, 2] = -1e-4 * (1 + rng.random(x.shape[0]))
    d[:, :2] = 1e-5 * rng.normal(size=(x.shape[0], 2))
    al = O.alpha_lin(x, sc.Y0, d)
    assert 0 < al < np.inf
    E = O.lagged(x, sc.Y0, d, [al, al / 0.9 * (1 - 1e-9), al / 0.9 * (1 + 1e-9)])
    assert np.isfinite(E[0]) and np.isfinite(E[1]) and np.isinf(E[2])
    # a direction that opens every gap gives no bound
    assert O.alpha_lin(x, sc.Y0, -d) == np.inf


def test_face_sample_geometry_direct(oracle_mod):
    # the exported face samples satisfy Eq. (gap) with the hit point inside
    # the master triangle; beta^m recomputed by a least-squares projection
    sc, x = small_indent(L=1)
    O = oracle_mod.Scene(sc)
    smp = O.samples(x, sc.Y0)
    face = smp[smp[:, 0] == 2]
    assert face.shape[0] > 10
    for row in face[:50]:
        s, m, g = int(row[1]), int(row[2]), row[3]
        bs = row[8:11]
        T = x[sc.stris[s]]
        n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
        xs = bs @ T
        p = xs + g * n
        Y = sc.Y0[sc.mtris[m]]
        A = np.stack([Y[1] - Y[0], Y[2] - Y[0]], axis=1)
        vw, *_ = np.linalg.lstsq(A, p - Y[0], rcond=None)
        assert np.linalg.norm(A @ vw - (p - Y[0])) < 1e-12
        assert min(1 - vw.sum(), vw[0], vw[1]) >= -1e-12
        assert 0 < g < row[4]
