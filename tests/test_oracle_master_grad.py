"""Pins of the oracle's master rows (orc_master_grad: the gradient of the
GMCP potential with respect to the master vertices, Sec. 4.3 with Eq. gap)
against finite differences where the frozen-normal gradient is exact, and
against the balance of forces and torques with the slave rows."""
import numpy as np
import pytest

from helpers import flat_over_big_triangle, small_indent


@pytest.mark.parametrize("L", [1, 2])
def test_flat_master_rows_match_finite_differences(oracle_mod, L):
    # Flat pad (normal -z) over one large parallel master triangle, far from
    # its edges (gamma = 1).  Moving a master vertex along z tilts the master
    # plane: each gap changes by -beta^m_j dz at first order and the hit
    # points keep their barycentrics, so dPsi/dz_j is exact.  An in-plane
    # move leaves every gap unchanged: dPsi/dx_j = dPsi/dy_j = 0.
    sc, x, xm = flat_over_big_triangle(nq=3, gap=3e-5, L=L)
    O = oracle_mod.Scene(sc)
    gm = O.master_grad(x, xm)
    assert np.all(np.abs(gm[:, :2]) == 0.0)
    h = 1e-10
    for j in range(3):
        for c in range(3):
            p, m = xm.copy(), xm.copy()
            p[j, c] += h
            m[j, c] -= h
            fd = (O.contact(x, p)["energy"] - O.contact(x, m)["energy"]) / (2 * h)
            scale = np.abs(gm).max()
            assert abs(fd - gm[j, c]) < 1e-6 * scale, (j, c, fd, gm[j, c])
    # and the sum over the master is the closed form kappa A B'(g) (+z)
    B, dB, _ = oracle_mod.barrier(3e-5, sc.params["dhat"])
    np.testing.assert_allclose(gm.sum(axis=0), [0, 0, -sc.params["kappa"] * (3e-3) ** 2 * dB],
                               rtol=1e-12, atol=1e-30)


@pytest.mark.parametrize("L,subdiv", [(1, 2), (2, 3)])
def test_master_rows_balance_slave_rows(oracle_mod, L, subdiv):
    # Every sample pushes its slave point and its master point with equal and
    # opposite forces along n_s (both weight sets sum to one), and x_m - x_s
    # is parallel to n_s: the net force and the net torque of slave and
    # master rows together vanish.  Face, edge and point samples all occur.
    sc, x = small_indent(n_quads=10, subdiv=subdiv, press=0.15e-3, L=L)
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    assert all(n > 0 for n in r["n_samples"])
    gs, gm = r["grad"], O.master_grad(x, sc.Y0)
    f = np.abs(gs).sum()
    np.testing.assert_allclose(gm.sum(axis=0), -gs.sum(axis=0), rtol=0, atol=1e-12 * f)
    torque = np.cross(sc.Y0, gm).sum(axis=0) + np.cross(x, gs).sum(axis=0)
    lever = max(np.abs(x).max(), np.abs(sc.Y0).max())
    assert np.abs(torque).max() < 1e-10 * f * lever
    # the master rows are not the slave rows moved over: a torque-free check
    # with the slave barycentrics in place of the master ones would fail
    assert np.abs(gm).max() > 0


def test_no_contact_gives_zero_master_rows(oracle_mod):
    sc, x, xm = flat_over_big_triangle(nq=2, gap=2e-4)   # beyond dhat = 1e-4
    O = oracle_mod.Scene(sc)
    assert np.all(O.master_grad(x, xm) == 0.0)


def test_flat_master_blocks_match_finite_differences(oracle_mod):
    # Same parallel-plane scene: the master rows and the slave rows are exact
    # there, so their derivatives with respect to a master vertex are the
    # master-master and slave-master blocks.  Along the normal (z) the
    # Gauss-Newton form is exact.  An in-plane move of a master vertex
    # changes no gap but does change the master weights bm_j of the cast
    # points, a term B'(g) dbm_j/dy that the Gauss-Newton form leaves out
    # (as the slave side leaves out its own weight derivatives), so the
    # master-master blocks are compared on their z column only.
    sc, x, xm = flat_over_big_triangle(nq=3, gap=3e-5, L=1)
    O = oracle_mod.Scene(sc)
    nv = x.shape[0]
    H = O.master_hess(x, xm)
    assert H
    h = 1e-10
    fd_m = np.zeros((3, 3, 3, 3))            # [row master j][col master i][p][q]
    fd_s = np.zeros((nv, 3, 3, 3))           # [slave a][col master i][p][q]
    for i in range(3):
        for q in range(3):
            p_, m_ = xm.copy(), xm.copy()
            p_[i, q] += h
            m_[i, q] -= h
            fd_m[:, i, :, q] = (O.master_grad(x, p_) - O.master_grad(x, m_)) / (2 * h)
            fd_s[:, i, :, q] = (O.contact(x, p_)["grad"] - O.contact(x, m_)["grad"]) / (2 * h)
    scale = max(np.abs(b).max() for b in H.values())
    for j in range(3):
        for i in range(3):
            np.testing.assert_allclose(H.get((nv + j, nv + i), np.zeros((3, 3)))[:, 2], fd_m[j, i][:, 2],
                                       rtol=0, atol=1e-6 * scale)
            # the in-plane columns of the exact derivative are the weight term
            assert np.abs(fd_m[j, i][:, :2]).max() < 1e-3 * scale
    for a in range(nv):
        for i in range(3):
            np.testing.assert_allclose(H.get((a, nv + i), np.zeros((3, 3))), fd_s[a, i],
                                       rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("L,subdiv", [(1, 2), (2, 3)])
def test_joint_hessian_annihilates_translations(oracle_mod, L, subdiv):
    # Moving slave and master together changes no gap, so every block row of
    # the joint Hessian (slave-slave from the contact evaluation, slave-master
    # and its transpose, master-master) sums to zero.
    sc, x = small_indent(n_quads=10, subdiv=subdiv, press=0.15e-3, L=L)
    O = oracle_mod.Scene(sc)
    r = O.contact(x, sc.Y0)
    H = O.master_hess(x, sc.Y0)
    rows = {}
    def add(u, b):
        rows[u] = rows.get(u, np.zeros((3, 3))) + b
    for (u, v), b in zip(r["blk_ij"], r["blk"]):
        add(int(u), b)
    nv = x.shape[0]
    for (u, v), b in H.items():
        add(u, b)
        if u < nv:          # slave-master: its transpose is the master-slave block
            add(v, b.T)
    scale = max(np.abs(b).max() for b in r["blk"])
    assert any(u >= nv for u in rows)
    for u, b in rows.items():
        assert np.abs(b).max() < 1e-10 * scale, (u, b)
