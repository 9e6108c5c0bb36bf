"""Pins of the oracle's dual-mesh mapper (Sec. 3.2, Eqs. bary_proj, decomp,
gram, bary_interp) against what the mathematics fixes: coordinates built
from chosen (u, v, w, delta), the identity on the undeformed mesh, rigid
invariance, the nearest triangle of points above a flat grid, and the
quadratic convergence of the interpolation error under a smooth bend."""
import numpy as np
import pytest

from oracle import oracle as O


def grid_mesh(n, size=1.0):
    """Flat n x n quad grid in z = 0, two triangles per quad (normal +z)."""
    xs = np.linspace(0.0, size, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    T = []
    for i in range(n):
        for j in range(n):
            a, b = i * (n + 1) + j, (i + 1) * (n + 1) + j
            T += [[a, b, b + 1], [a, b + 1, a + 1]]
    return V, np.array(T, dtype=np.int32)


def test_coords_recover_chosen_values():
    rng = np.random.default_rng(3)
    for _ in range(200):
        v0, v1, v2 = rng.normal(size=(3, 3))
        n = np.cross(v1 - v0, v2 - v0)
        n /= np.linalg.norm(n)
        u, v = rng.uniform(-0.5, 1.5, 2)
        w = 1.0 - u - v
        delta = rng.uniform(-1, 1)
        p = u * v0 + v * v1 + w * v2 + delta * n
        np.testing.assert_allclose(O.dual_map_coords(p, v0, v1, v2), [u, v, w, delta], rtol=0, atol=1e-11)


def test_undeformed_identity_and_rigid_invariance():
    rng = np.random.default_rng(4)
    V, T = grid_mesh(6)
    V = V + np.c_[np.zeros((len(V), 2)), 0.05 * np.sin(3 * V[:, 0]) * np.cos(2 * V[:, 1])]
    P = np.c_[rng.uniform(-0.1, 1.1, (300, 2)), rng.uniform(-0.2, 0.2, 300)]
    tri, uvwd, _ = O.dual_map_build(V, T, P)
    np.testing.assert_allclose(O.dual_map_apply(V, T, tri, uvwd), P, rtol=0, atol=1e-12)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    t = np.array([0.3, -2.0, 5.0])
    np.testing.assert_allclose(O.dual_map_apply(V @ R.T + t, T, tri, uvwd), P @ R.T + t, rtol=0, atol=1e-12)


def test_nearest_triangle_above_flat_grid():
    rng = np.random.default_rng(5)
    V, T = grid_mesh(8)
    P = np.c_[rng.uniform(0.01, 0.99, (400, 2)), rng.uniform(-0.3, 0.3, 400)]
    tri, uvwd, d2 = O.dual_map_build(V, T, P)
    # the chosen triangle contains the point's projection, the offset is the height
    assert (uvwd[:, :3] >= -1e-12).all()
    np.testing.assert_allclose(uvwd[:, 3], P[:, 2], rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.sqrt(d2), np.abs(P[:, 2]), rtol=0, atol=1e-14)
    # a point outside the grid maps to its nearest corner triangle
    tri2, uvwd2, d22 = O.dual_map_build(V, T, np.array([[1.3, 1.4, 0.0]]))
    assert np.isclose(d22[0], 0.3 ** 2 + 0.4 ** 2)
    assert (T[tri2[0]] == 80).any()   # vertex (8, 8) of the 9 x 9 grid


@pytest.mark.parametrize("n", [8])
def test_interpolation_error_is_quadratic(n):
    """A smooth bend of the simulation surface: the mapped visual points
    approach the bent surface with an error that quarters when h halves
    (the O(h^2) statement of Sec. 3.2)."""
    rng = np.random.default_rng(6)
    P = np.c_[rng.uniform(0.05, 0.95, (500, 2)), np.zeros(500)]

    def bend(X):
        k = 0.8
        return np.c_[X[:, 0], X[:, 1], 0.5 * k * (X[:, 0] - 0.5) ** 2 + 0.3 * np.sin(2 * X[:, 1])]

    errs = []
    for m in (n, 2 * n, 4 * n):
        V, T = grid_mesh(m)
        tri, uvwd, _ = O.dual_map_build(V, T, P)
        Q = O.dual_map_apply(bend(V), T, tri, uvwd)
        errs.append(np.abs(Q - bend(P)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, errs
