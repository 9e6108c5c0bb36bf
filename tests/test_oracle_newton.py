"""Pins of the oracle's elasticity, linear solver and time step (reading R7/R8
of the IPC problem statement, Sec. 2.1)."""
import numpy as np
import pytest

from paper_2605_24339_b300 import scenes as S


def _tet(rng, scale=1e-3):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float) * scale
    X += rng.normal(size=X.shape) * 0.1 * scale
    Dm = (X[1:] - X[0]).T
    return X, np.linalg.inv(Dm), abs(np.linalg.det(Dm)) / 6


MU, LAM = 1e5, 1e6


def test_nh_rest(oracle_mod):
    X, Dmi, V = _tet(np.random.default_rng(0))
    ok, psi, g, H = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, X)
    assert ok and abs(psi) < 1e-20 and np.abs(g).max() < 1e-12 * MU * V / 1e-3


def _nh_exact(Dmi, V, X, x, mu, lam, dps=60):
    """The textbook energy mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2 with
    F = Ds Dm^-1, evaluated in 60-digit arithmetic (mpmath) from the same
    FP64 inputs."""
    import mpmath as mp
    mp.mp.dps = dps
    Xm = [[mp.mpf(float(v)) for v in row] for row in np.asarray(X).reshape(4, 3)]
    xm = [[mp.mpf(float(v)) for v in row] for row in np.asarray(x).reshape(4, 3)]
    Dm = mp.matrix(3, 3)
    Ds = mp.matrix(3, 3)
    for r in range(3):
        for c in range(3):
            Dm[r, c] = Xm[c + 1][r] - Xm[0][r]
            Ds[r, c] = xm[c + 1][r] - xm[0][r]
    F = Ds * mp.inverse(Dm)
    Ic = sum(F[i, j] ** 2 for i in range(3) for j in range(3))
    lnJ = mp.log(mp.det(F))
    vol = abs(mp.det(Dm)) / 6
    return float(vol * (mu / 2 * (Ic - 3) - mu * lnJ + lam / 2 * lnJ ** 2))


@pytest.mark.parametrize("strain", [1e-8, 1e-6, 1e-4, 1e-2, 0.3])
def test_nh_energy_relative_precision(oracle_mod, strain):
    """Reading R15: the oracle's energy keeps ~1e-12 relative precision of
    the energy itself down to tiny strains (the textbook FP64 evaluation
    loses ~1e-16 / strain^2 of it), pinned against 60-digit arithmetic."""
    rng = np.random.default_rng(11)
    X, Dmi, V = _tet(rng)
    for _ in range(4):
        x = X + strain * 1e-3 * rng.normal(size=X.shape)
        ok, psi, _, _ = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x)
        ref = _nh_exact(Dmi, V, X, x, MU, LAM)
        assert ok and ref > 0
        # H = (Ds - Dm) Dm^-1 with the FP64 Dm^-1 is H times (1 + O(1e-16)),
        # so the energy (quadratic in H) stays accurate relative to itself
        assert psi == pytest.approx(ref, rel=1e-12)


def test_nh_gradient_fd(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(5):
        X, Dmi, V = _tet(rng)
        x = X + rng.normal(size=X.shape) * 2e-4
        ok, psi, g, H = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x)
        assert ok
        h = 1e-9
        for i in range(12):
            e = np.zeros(12); e[i] = h
            p = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x.ravel() + e)[1]
            m = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x.ravel() - e)[1]
            assert (p - m) / (2 * h) == pytest.approx(g[i], rel=1e-5, abs=1e-9 * np.abs(g).max())


def test_nh_hessian_fd_stretch(oracle_mod):
    # under a pure stretch (F = diag(s), s > 1) every eigenvalue of dP/dF is
    # positive (twist modes mu - (mu - lam ln J)/(s_i s_j) > 0), so the
    # projection is the identity and the Hessian is the derivative of the
    # gradient.  (At rest the twist modes are exactly zero.)
    rng = np.random.default_rng(2)
    X, Dmi, V = _tet(rng)
    x = (X @ np.diag([1.01, 1.02, 1.015]).T).ravel()
    ok, psi, g, H = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x)
    h = 1e-10
    for i in range(12):
        e = np.zeros(12); e[i] = h
        gp = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x + e)[2]
        gm = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x - e)[2]
        np.testing.assert_allclose((gp - gm) / (2 * h), H[:, i], rtol=1e-5,
                                   atol=1e-6 * np.abs(H).max())


def test_nh_hessian_psd_large_strain(oracle_mod):
    rng = np.random.default_rng(3)
    X, Dmi, V = _tet(rng)
    # strong stretch makes dP/dF indefinite; the projected Hessian is PSD
    x = X.copy(); x[:, 0] *= 2.5
    ok, psi, g, H = oracle_mod.nh_tet(Dmi, V, MU, LAM, X, x)
    assert ok
    w = np.linalg.eigvalsh(H)
    assert w.min() >= -1e-9 * w.max()
    # inverted tet is rejected
    xi = X.copy(); xi[3, 2] = -xi[3, 2] - 1e-3
    assert not oracle_mod.nh_tet(Dmi, V, MU, LAM, X, xi)[0]


def test_psd_projection_matches_eigh(oracle_mod):
    rng = np.random.default_rng(4)
    for n in (3, 9, 12):
        A = rng.normal(size=(n, n)); A = A + A.T
        P = oracle_mod.psd_project(A)
        w, V = np.linalg.eigh(A)
        ref = (V * np.maximum(w, 0)) @ V.T
        np.testing.assert_allclose(P, ref, rtol=0, atol=1e-12 * np.abs(A).max())
        # idempotent on PSD input
        np.testing.assert_allclose(oracle_mod.psd_project(ref), ref, rtol=0, atol=1e-12 * np.abs(A).max())


def _small_sim(oracle_mod, n_quads=6, subdiv=1, press=0.1e-3, n_steps=4, radius=5e-3, **kw):
    sc = S.tactile_indent(n_quads=n_quads, side=n_quads * 0.5e-3, nz=2, thick=1e-3,
                          sphere_subdiv=subdiv, radius=radius, press=press, n_steps=n_steps)
    sc.params.update(kw)
    O = oracle_mod.Scene(sc)
    return sc, O, oracle_mod.Sim(O)


def test_pcg_matches_dense_solve(oracle_mod):
    sc, O, sim = _small_sim(oracle_mod)
    x = S.drape_on_master(sc, 0.05e-3)
    v = np.zeros_like(x)
    ok, E, G, A = sim.system(x, v)
    assert ok
    rp, ci = sim.pattern()
    n = 3 * x.shape[0]
    Ad = np.zeros((n, n))
    for i in range(x.shape[0]):
        for k in range(rp[i], rp[i + 1]):
            Ad[3 * i:3 * i + 3, 3 * ci[k]:3 * ci[k] + 3] = A[k]
    np.testing.assert_allclose(Ad, Ad.T, rtol=0, atol=1e-12 * np.abs(Ad).max())
    assert np.linalg.eigvalsh(Ad).min() > 0
    b = -G.ravel()
    ref = np.linalg.solve(Ad, b)
    got, it = sim.pcg(A, b, tol=1e-13)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def _flat_press_sim(oracle_mod, nq=4, n_steps=4):
    """pad pressed by its top face onto one large flat master triangle"""
    from helpers import flat_press
    sc = flat_press(nq=nq, n_steps=n_steps)
    O = oracle_mod.Scene(sc)
    return sc, O, oracle_mod.Sim(O)


@pytest.mark.parametrize("case", ["flat", "sphere"])
def test_newton_steps_converge_and_stay_feasible(oracle_mod, case):
    if case == "flat":
        sc, O, sim = _flat_press_sim(oracle_mod)
        n_steps = sc.n_steps
    else:
        sc, O, sim = _small_sim(oracle_mod, n_quads=8, subdiv=3, press=0.2e-3, n_steps=6,
                                pcg_rel_tol=1e-6)
        n_steps = 3
    x = sc.X.copy()
    v = sc.v_dirichlet.copy()
    for step in range(n_steps):
        x_new, v_new, st = sim.step(x, v)
        assert st.status == 0, st.status
        assert st.residual <= 1e-6
        # every tet stays positively oriented
        a = x_new[sc.tets[:, 1]] - x_new[sc.tets[:, 0]]
        b = x_new[sc.tets[:, 2]] - x_new[sc.tets[:, 0]]
        c = x_new[sc.tets[:, 3]] - x_new[sc.tets[:, 0]]
        assert np.einsum("ij,ij->i", np.cross(a, b), c).min() > 0
        # Dirichlet vertices follow their script
        top = sc.dirichlet.astype(bool)
        np.testing.assert_allclose(x_new[top], x[top] + sc.params["h"] * v[top], rtol=0, atol=1e-15)
        x, v = x_new, v_new
        v[top] = sc.v_dirichlet[top]
    # the pad reached the master: contact energy is present
    assert O.contact(x, O.sc.Y0)["energy"] > 0


def test_newton_zero_motion_is_stationary(oracle_mod):
    sc, O, sim = _small_sim(oracle_mod)
    x = sc.X.copy()
    v = np.zeros_like(x)
    x_new, v_new, st = sim.step(x, v)
    assert st.status == 0 and st.newton_iters <= 1
    np.testing.assert_allclose(x_new, x, rtol=0, atol=1e-14)
