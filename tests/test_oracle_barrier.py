"""Pins of the oracle's closed forms: Hermite step (Sec. 4.3), IPC barrier
(Sec. 4.2) and the fixed face rule (reading R1 of Sec. 4.1)."""
import numpy as np
import pytest

from helpers import load_golden


def test_hermite_golden(oracle_mod):
    for x, delta, H in load_golden("hermite_smoothstep.txt"):
        assert oracle_mod.hermite(x, delta) == pytest.approx(H, abs=1e-15)


def test_hermite_c1(oracle_mod):
    # C1: one-sided derivatives vanish at 0 and delta, and H'(delta/2) = 1.5/delta
    d, h = 0.1, 1e-7
    H = oracle_mod.hermite
    # one-sided differences of a function with H'' = 6/delta^2 at the ends
    assert (H(h, d) - H(0, d)) / h == pytest.approx(0.0, abs=4 * h / d ** 2)
    assert (H(d, d) - H(d - h, d)) / h == pytest.approx(0.0, abs=4 * h / d ** 2)
    assert (H(d / 2 + h, d) - H(d / 2 - h, d)) / (2 * h) == pytest.approx(1.5 / d, rel=1e-7)
    xs = np.linspace(-0.05, 0.15, 401)
    v = np.array([H(x, d) for x in xs])
    assert np.all(np.diff(v) >= 0)


def test_barrier_vanishes_at_support(oracle_mod):
    for eps in (1e-5, 1e-4, 3e-3):
        B, dB, d2B = oracle_mod.barrier(eps, eps)
        assert (B, dB, d2B) == (0.0, 0.0, 0.0)
        B, dB, d2B = oracle_mod.barrier(2 * eps, eps)
        assert (B, dB, d2B) == (0.0, 0.0, 0.0)
        # C2 continuity at eps from below
        B, dB, d2B = oracle_mod.barrier(eps * (1 - 1e-6), eps)
        assert abs(B) < 1e-15 * eps ** 2 + 1e-30
        assert abs(dB) < 1e-10 * eps
        assert abs(d2B) < 1e-4


def test_barrier_derivatives_fd(oracle_mod):
    eps = 1e-4
    for g in np.linspace(0.02, 0.98, 13) * eps:
        h = eps * 1e-6
        Bp, dBp, _ = oracle_mod.barrier(g + h, eps)
        Bm, dBm, _ = oracle_mod.barrier(g - h, eps)
        B, dB, d2B = oracle_mod.barrier(g, eps)
        assert (Bp - Bm) / (2 * h) == pytest.approx(dB, rel=1e-7)
        assert (dBp - dBm) / (2 * h) == pytest.approx(d2B, rel=1e-7)
        assert B > 0 and dB < 0 and d2B > 0


def test_barrier_log_singularity(oracle_mod):
    eps = 1e-4
    B1, _, _ = oracle_mod.barrier(1e-3 * eps, eps)
    B2, _, _ = oracle_mod.barrier(1e-6 * eps, eps)
    # B ~ -eps^2 ln(g/eps) as g -> 0
    assert B1 == pytest.approx(-eps ** 2 * np.log(1e-3), rel=3e-3)
    assert B2 > B1
    B, dB, d2B = oracle_mod.barrier(0.0, eps)
    assert np.isinf(B)


def test_face_rule_golden(oracle_mod):
    ref = load_golden("face_rule_L1.txt")
    got = oracle_mod.face_rule(1)
    key = lambda a: np.lexsort(a.T[::-1])
    np.testing.assert_allclose(got[key(got)], ref[key(ref)], rtol=0, atol=1e-16)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_face_rule_properties(oracle_mod, L):
    b = oracle_mod.face_rule(L)
    assert b.shape == (4 ** L, 3)
    np.testing.assert_allclose(b.sum(axis=1), 1.0, atol=1e-15)
    assert np.all(b > 0)
    # exact for linear integrands: mean of the sample barycentrics is the centroid
    np.testing.assert_allclose(b.mean(axis=0), 1.0 / 3.0, atol=1e-15)
    assert len({tuple(np.round(r, 12)) for r in b}) == 4 ** L


def test_face_rule_quadratic_convergence(oracle_mod):
    # (1/A) int beta_0^2 dA = 1/6 and (1/A) int beta_0 beta_1 dA = 1/12; the
    # composite centroid rule errs by O(4^-L)
    errs = []
    for L in (1, 2, 3, 4):
        b = oracle_mod.face_rule(L)
        errs.append(abs(np.mean(b[:, 0] ** 2) - 1 / 6) + abs(np.mean(b[:, 0] * b[:, 1]) - 1 / 12))
    for a, c in zip(errs[:-1], errs[1:]):
        assert a / c == pytest.approx(4.0, rel=1e-6)
