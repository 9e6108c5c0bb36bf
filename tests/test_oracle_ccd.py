"""Pins of the oracle's distance routines and additive CCD (Li et al. 2021,
Alg. 1) against analytic times of impact, dense sampling and the
intersection-free invariant."""
import numpy as np
import pytest

from helpers import small_indent


def _tri_samples(t0, t1, t2, n=120):
    u, v = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n), indexing="ij")
    m = u + v <= 1
    u, v = u[m], v[m]
    return t0 + u[:, None] * (t1 - t0) + v[:, None] * (t2 - t0)


def test_point_triangle_distance_dense(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(20):
        t0, t1, t2, p = rng.normal(size=(4, 3))
        d2 = oracle_mod.pt_dist2(p, t0, t1, t2)
        q = _tri_samples(t0, t1, t2)
        brute = np.min(np.sum((q - p) ** 2, axis=1))
        assert d2 <= brute * (1 + 1e-12)
        assert np.sqrt(brute) - np.sqrt(d2) < 0.03 * (np.linalg.norm(t1 - t0) + np.linalg.norm(t2 - t0))


def test_edge_edge_distance_dense(oracle_mod):
    rng = np.random.default_rng(1)
    s = np.linspace(0, 1, 400)
    for _ in range(20):
        a0, a1, b0, b1 = rng.normal(size=(4, 3))
        d2 = oracle_mod.ee_dist2(a0, a1, b0, b1)
        P = a0 + s[:, None] * (a1 - a0)
        Q = b0 + s[:, None] * (b1 - b0)
        brute = np.min(np.sum((P[:, None, :] - Q[None, :, :]) ** 2, axis=2))
        assert d2 <= brute * (1 + 1e-12)
        assert np.sqrt(brute) - np.sqrt(d2) < 0.01 * max(np.linalg.norm(a1 - a0), np.linalg.norm(b1 - b0))
    # crossing skew lines at a known distance
    d2 = oracle_mod.ee_dist2([-1, 0, 0], [1, 0, 0], [0, -1, 0.25], [0, 1, 0.25])
    assert d2 == pytest.approx(0.0625, rel=1e-15)
    # parallel segments
    d2 = oracle_mod.ee_dist2([0, 0, 0], [1, 0, 0], [0.5, 0.3, 0], [2, 0.3, 0])
    assert d2 == pytest.approx(0.09, rel=1e-14)


@pytest.mark.parametrize("s", [0.1, 0.2, 0.5])
def test_accd_point_plane_analytic(oracle_mod, s):
    # point at height d above a large triangle moving toward it at speed v:
    # true TOI t* = d/v; the returned fraction is conservative and within the
    # slack: (1 - s) t* <= t <= t*
    for d, v in ((1e-4, 2e-4), (1e-3, 5e-3), (2e-5, 1e-3)):
        x = np.array([[0.1, 0.2, d], [-1, -1, 0], [3, -1, 0], [-1, 3, 0]])
        p = np.zeros((4, 3)); p[0, 2] = -v
        t, it = oracle_mod.accd(0, x, p, s=s)
        ts = d / v
        assert (1 - s) * ts * (1 - 1e-12) <= t <= ts
        # the triangle moving instead of the point gives the same answer
        p2 = np.zeros((4, 3)); p2[1:, 2] = v
        t2, _ = oracle_mod.accd(0, x, p2, s=s)
        assert (1 - s) * ts * (1 - 1e-12) <= t2 <= ts


def test_accd_edge_edge_analytic(oracle_mod):
    d, v = 3e-4, 1e-3
    x = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, d], [0, 1, d]], dtype=float)
    p = np.zeros((4, 3)); p[2:, 2] = -v
    t, _ = oracle_mod.accd(1, x, p, s=0.1)
    assert 0.9 * d / v * (1 - 1e-12) <= t <= d / v


def test_accd_no_collision(oracle_mod):
    x = np.array([[0.1, 0.2, 1e-3], [-1, -1, 0], [3, -1, 0], [-1, 3, 0]])
    p = np.zeros((4, 3))
    assert oracle_mod.accd(0, x, p)[0] == 1.0          # no motion
    p[0] = [1e-3, 0, 0]                                 # sliding parallel
    assert oracle_mod.accd(0, x, p)[0] == 1.0
    p[0] = [0, 0, +1e-3]                                # moving away
    assert oracle_mod.accd(0, x, p)[0] == 1.0
    p[0] = [0, 0, -0.5e-3]                              # stops at half the gap
    assert oracle_mod.accd(0, x, p)[0] == 1.0


def _min_distance(sc, x, xm):
    """brute-force min distance between the slave surface and the master"""
    S, M = sc.stris, sc.mtris
    best = np.inf
    sv = np.unique(S)
    mv = np.unique(M)
    for v in sv:
        for t in M:
            best = min(best, np.sqrt(max(0.0, _pt(x[v], xm[t]))))
    for v in mv:
        for t in S:
            best = min(best, np.sqrt(max(0.0, _pt(xm[v], x[t]))))
    return best


_oracle = None


def _pt(p, T):
    return _oracle.pt_dist2(p, T[0], T[1], T[2])


def test_ccd_keeps_trajectory_intersection_free(oracle_mod):
    global _oracle
    _oracle = oracle_mod
    sc, x = small_indent(n_quads=4, subdiv=1, press=0.05e-3)
    O = oracle_mod.Scene(sc)
    rng = np.random.default_rng(5)
    for trial in range(3):
        dx = np.zeros_like(x)
        dx[:, 2] = -(3e-4 + 2e-4 * rng.random(x.shape[0]))
        dx[:, :2] = 5e-5 * rng.normal(size=(x.shape[0], 2))
        a, al, aa = O.ccd_max_step(x, dx, sc.Y0)
        assert 0 < a < 1 and a == min(1.0, al, aa)
        for f in np.linspace(0, 1, 33)[1:]:
            assert _min_distance(sc, x + f * a * dx, sc.Y0) > 0
        # the full step does intersect (so CCD did something)
        assert _min_distance(sc, x + dx, sc.Y0) < 1e-4 or a < 1


def test_accd_min_matches_pairwise(oracle_mod):
    # the env-wide minimum equals the minimum of single-pair calls over the
    # swept-box candidates (no pair is dropped)
    sc, x = small_indent(n_quads=3, subdiv=1, press=0.02e-3)
    O = oracle_mod.Scene(sc)
    dx = np.zeros_like(x); dx[:, 2] = -4e-4
    al, info = O.accd_min(x, dx, sc.Y0)
    assert info.n_pt > 0 and info.n_ee > 0 and 0 < al < 1
    best = 1.0
    sv = np.unique(sc.stris)
    for v in sv:
        for t in sc.mtris:
            X4 = np.vstack([x[v], sc.Y0[t]]); P4 = np.vstack([dx[v], np.zeros((3, 3))])
            best = min(best, oracle_mod.accd(0, X4, P4)[0])
    assert al <= best


def test_surface_min_dist_closed_forms(oracle_mod):
    """The brute-force surface distance (used by the CCD stress checks) on
    configurations with a known answer: parallel faces, a vertex over a
    face interior, and two crossing edges whose closest points are interior
    to both."""
    h = 0.37
    A = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    B = A + [0, 0, h]
    T = np.array([[0, 1, 2]], dtype=np.int32)
    assert oracle_mod.surface_min_dist(A, T, B, T) == pytest.approx(h, rel=1e-14)
    # a tilted triangle whose lowest vertex sits h above the interior of A
    C = np.array([[0.25, 0.25, h], [2.0, 2.0, 3.0], [-1.0, 3.0, 2.0]])
    assert oracle_mod.surface_min_dist(A, T, C, T) == pytest.approx(h, rel=1e-14)
    assert oracle_mod.surface_min_dist(C, T, A, T) == pytest.approx(h, rel=1e-14)
    # edge along x at z = 0 against edge along y at z = h, both tris turned away
    D = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, -1]], dtype=np.float64)
    E = np.array([[0, -1, h], [0, 1, h], [1, 0, h + 1]], dtype=np.float64)
    assert oracle_mod.surface_min_dist(D, T, E, T) == pytest.approx(h, rel=1e-14)
    # every vertex is farther than h: the minimum is the edge-edge distance
    vmin = min(np.sqrt(oracle_mod.pt_dist2(p, *E)) for p in D)
    assert vmin > 1.2 * h


def test_thin_shell_is_closed_and_outward():
    from paper_2605_24339_b300 import scenes as S
    from collections import Counter
    Y, F = S.thin_shell(5, 4e-3, 1e-3)
    E = Counter()
    for t in F:
        for k in range(3):
            E[(int(t[k]), int(t[(k + 1) % 3]))] += 1
    assert all(c == 1 for c in E.values())
    assert all(E[(b, a)] == 1 for (a, b) in E)            # every edge shared, opposite directions
    vol = sum(np.dot(Y[t[0]], np.cross(Y[t[1]], Y[t[2]])) for t in F) / 6.0
    assert vol == pytest.approx(4e-3 * 4e-3 * 1e-3, rel=1e-12)   # outward normals
