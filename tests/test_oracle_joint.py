"""The oracle's time step with a deformable master (Sec. 4.2-4.3 with
Eq. gap: every sample's gap gradient is bm_j n_s on master vertex j), pinned
by what the mechanics fixes rather than by the formulas themselves:

- the contact patch test (Sec. 5.1, "Contact patch test", Table
  patch_test): two blocks of 1 x 1 x 0.5 on non-matching meshes, E = 1000,
  nu = 0, a pressure of 10 on the top: the exact static state is
  sigma_zz = -10 in both blocks.  The mean must hold to 2e-3 in each block
  (it is the load over the area, transmitted through the master rows); the
  largest error of a single tet is reported against the paper's table and
  bounded by the order of magnitude only (its meshes are not available);
- action and reaction: without Dirichlet vertices or external forces, the
  joint gradient sums to M (x - xhat) over all vertices (elastic and contact
  forces cancel);
- translation invariance of the joint matrix: A t = M t for a rigid
  translation t (the elastic and contact blocks, slave-slave, slave-master
  and master-master, annihilate it).

A wrong sign of the master rows fails the second pin, and a wrong sign or a
missing transpose of the slave-master blocks the third (checked by planting
each in a scratch copy)."""
import numpy as np
import pytest

from helpers import patch_report
from paper_2605_24339_b300 import scenes as S


def _contact_state(sc, lower=0.0016, seed=0):
    n = sc.X.shape[0]
    x = np.concatenate([sc.X, sc.Y0])
    x[:n, 2] -= lower
    x[:n] += 1e-5 * np.random.default_rng(seed).normal(size=(n, 3))
    return x


def test_patch_test_oracle(oracle_mod):
    sc, f = S.patch_test(kappa=1e4, h=0.05, density=1.0)
    sim = oracle_mod.Sim(oracle_mod.Scene(sc))
    sim.set_fext(f)
    x = np.concatenate([sc.X, sc.Y0])
    v = np.zeros_like(x)
    for step in range(12):
        x, v, st = sim.step(x, v)
        assert st.status in (0, 5), (step, st.status)
    assert st.status == 0
    rep = patch_report(sc, x)
    print("patch test (oracle, kappa 1e4):", rep)
    for blk in ("upper", "lower"):
        assert rep[blk]["mean"] == pytest.approx(-10.0, rel=2e-3)
        assert rep[blk]["max_rel_err"] < 0.1
        assert rep[blk]["spurious"] < 1.0
    # the blocks stay separated, within the barrier's support
    n = sc.X.shape[0]
    gap = x[:n][sc.stris.ravel(), 2].min() - x[n:, 2].max()
    assert 0.0 < gap < sc.params["dhat"]


@pytest.fixture
def free_joint(oracle_mod):
    sc, _ = S.patch_test(kappa=1e4, h=0.05, density=1.0)
    sc.mdirichlet = np.zeros(sc.Y0.shape[0], dtype=np.uint8)
    return sc, oracle_mod.Sim(oracle_mod.Scene(sc))


def test_joint_forces_balance(free_joint):
    sc, sim = free_joint
    x = _contact_state(sc)
    v = np.zeros_like(x)
    ok, E, G, A = sim.system(x, v)
    assert ok and E > 0
    # contact is active: the contact forces are a visible part of G
    assert np.abs(G).max() > 1e-3
    assert np.abs(G.sum(axis=0)).max() < 1e-12 * np.abs(G).max()


def test_joint_matrix_annihilates_translations(free_joint):
    sc, sim = free_joint
    x = _contact_state(sc)
    ok, E, G, A = sim.system(x, np.zeros_like(x))
    assert ok
    rp, ci = sim.pattern()
    m = sim.mass()
    for t in (np.array([1.0, 0, 0]), np.array([0, 0, 1.0]), np.array([0.3, -0.2, 0.9])):
        y = np.zeros((x.shape[0], 3))
        for i in range(x.shape[0]):
            y[i] = (A[rp[i]:rp[i + 1]] @ t).sum(axis=0)
        ref = m[:, None] * t[None, :]
        assert np.abs(y - ref).max() < 1e-10 * np.abs(ref).max()
