"""Pins of the oracle's paper-exact face sampler (Sec. 4.1 "Face samples":
projection onto the slave tangent plane, Sutherland-Hodgman clip, fan
triangulation, 3-point Gauss per sub-triangle; reading R18) against what
geometry fixes: full-cover and contained overlaps, the closed-form overlap
of a shifted right triangle, exact integration of quadratics (checked with
the independent edge-midpoint rule), samples inside both triangles, exact
gaps to a tilted plane, and overlap areas of random pairs against a fine
point-in-triangle count."""
import numpy as np
import pytest

from oracle import oracle as O

S0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


def cross2(a, b):
    return a[0] * b[1] - a[1] * b[0]


def xs_of(smp, xs):
    return smp[:, :3] @ xs


def test_slave_inside_master_gives_the_slave_area_and_exact_gaps():
    # a tilted master plane z = 0.3 + 0.1 x - 0.2 y covering the slave
    def zf(x, y):
        return 0.3 + 0.1 * x - 0.2 * y
    xm = np.array([[-2, -2, zf(-2, -2)], [4, -2, zf(4, -2)], [-2, 4, zf(-2, 4)]], dtype=float)
    smp = O.face_clip_samples(S0, xm)
    assert len(smp) == 3
    np.testing.assert_allclose(smp[:, 7].sum(), 0.5, rtol=1e-14)
    p = xs_of(smp, S0)
    np.testing.assert_allclose(smp[:, 6], zf(p[:, 0], p[:, 1]), rtol=0, atol=1e-14)
    hit = smp[:, 3:6] @ xm
    np.testing.assert_allclose(hit, p + smp[:, 6:7] * np.array([0, 0, 1.0]), rtol=0, atol=1e-13)


def test_master_inside_slave_gives_the_master_projected_area():
    big = 4.0 * S0 - np.array([0.5, 0.5, 0.0])
    xm = np.array([[0.2, 0.2, 0.7], [0.9, 0.3, 0.5], [0.3, 0.8, 0.6]])
    smp = O.face_clip_samples(big, xm)
    a = 0.5 * abs(cross2(xm[1, :2] - xm[0, :2], xm[2, :2] - xm[0, :2]))
    np.testing.assert_allclose(smp[:, 7].sum(), a, rtol=1e-14)
    assert (smp[:, :3] >= -1e-14).all() and (smp[:, 3:6] >= -1e-12).all()


@pytest.mark.parametrize("s", [0.1, 0.35, 0.8])
def test_shifted_triangle_overlap_and_quadratic_exactness(s):
    xm = S0 + np.array([s, 0.0, 0.25])
    smp = O.face_clip_samples(S0, xm)
    # the overlap is the triangle (s, 0), (1, 0), (s, 1 - s)
    np.testing.assert_allclose(smp[:, 7].sum(), 0.5 * (1 - s) ** 2, rtol=1e-13)
    T = np.array([[s, 0.0], [1.0, 0.0], [s, 1.0 - s]])
    f = lambda p: 1.0 + 2.0 * p[..., 0] - 0.5 * p[..., 1] + 3.0 * p[..., 0] ** 2 - p[..., 0] * p[..., 1] + 0.7 * p[..., 1] ** 2
    mids = np.array([(T[0] + T[1]) / 2, (T[1] + T[2]) / 2, (T[2] + T[0]) / 2])
    exact = 0.5 * (1 - s) ** 2 / 3.0 * f(mids).sum()
    p = xs_of(smp, S0)[:, :2]
    np.testing.assert_allclose((smp[:, 7] * f(p)).sum(), exact, rtol=1e-13)
    np.testing.assert_allclose(smp[:, 6], 0.25, rtol=0, atol=1e-14)


def point_in_tri(P, T):
    d = lambda a, b, p: (b[0] - a[0]) * (p[..., 1] - a[1]) - (b[1] - a[1]) * (p[..., 0] - a[0])
    s = [d(T[0], T[1], P), d(T[1], T[2], P), d(T[2], T[0], P)]
    return ((s[0] >= 0) & (s[1] >= 0) & (s[2] >= 0)) | ((s[0] <= 0) & (s[1] <= 0) & (s[2] <= 0))


def test_random_overlap_area_against_a_fine_count():
    rng = np.random.default_rng(8)
    g = (np.arange(1200) + 0.5) / 1200 * 3.0 - 1.0
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([X, Y], -1)
    cell = (3.0 / 1200) ** 2
    n_checked = 0
    for _ in range(12):
        xs = np.c_[rng.uniform(-0.5, 1.5, (3, 2)), np.zeros(3)]
        xm = np.c_[rng.uniform(-0.5, 1.5, (3, 2)), rng.uniform(0.1, 0.4, 3)]
        if abs(cross2(xs[1, :2] - xs[0, :2], xs[2, :2] - xs[0, :2])) < 0.2:
            continue
        if np.cross(xs[1] - xs[0], xs[2] - xs[0])[2] < 0:
            xs = xs[[0, 2, 1]]
        smp = O.face_clip_samples(xs, xm)
        count = (point_in_tri(P, xs[:, :2]) & point_in_tri(P, xm[:, :2])).sum() * cell
        area = smp[:, 7].sum() if len(smp) else 0.0
        assert abs(area - count) < 2e-2 * max(count, 0.02), (area, count)
        if len(smp):
            assert (smp[:, :3] >= -1e-12).all() and (smp[:, 3:6] >= -1e-12).all()
        n_checked += 1
    assert n_checked >= 6
