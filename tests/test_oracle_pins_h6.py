"""Pins of the oracle's sixth-order variant (adjacent to the paper: the
sixth-order Hermite scheme of Nitadori & Makino 2008, the same block-timestep
procedure with snap), each against something other than its own formulas:
finite differences, closed forms of circular motion, polynomial exactness,
the scheme's error order."""
import math

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics


def test_snap_is_the_derivative_of_jerk_along_the_trajectories(orc):
    """Snap from force_snap against the central difference of the jerk
    (Eq. jrk, orc.force) along r(tau) = r + v tau + a tau^2/2, v(tau) =
    v + a tau, for arbitrary accelerations a: O(h^2) convergence."""
    n, eps = 24, 0.05
    m, r, v = ics.plummer(n, 61)
    rng = np.random.default_rng(5)
    a = rng.normal(size=(n, 3))
    _, _, snap, _ = orc.force_snap(m, r, v, a, eps)
    errs = []
    for h in (1e-4, 5e-5):
        jp = orc.force(m, r + v * h + a * h * h / 2, v + a * h, eps)[1]
        jm = orc.force(m, r - v * h + a * h * h / 2, v - a * h, eps)[1]
        fd = (jp - jm) / (2 * h)
        errs.append(np.max(np.abs(fd - snap)) / np.max(np.abs(snap)))
    assert errs[0] < 1e-5
    assert 3.0 < errs[0] / errs[1] < 5.0  # second order in h


def test_force_snap_acc_jerk_pot_are_eqs_acc_jrk_pot(orc):
    n, eps = 300, 4.0 / 300
    m, r, v = ics.plummer(n, 62)
    a_in = np.random.default_rng(1).normal(size=(n, 3))
    a, j, s, p = orc.force_snap(m, r, v, a_in, eps)
    a0, j0, p0 = orc.force(m, r, v, eps)
    assert np.max(np.abs(a - a0)) <= 1e-13 * np.max(np.abs(a0))
    assert np.max(np.abs(j - j0)) <= 1e-12 * np.max(np.abs(j0))
    assert np.max(np.abs(p - p0)) <= 1e-13 * np.max(np.abs(p0))


def test_snap_of_a_circular_binary(orc):
    """Two equal masses on a circular orbit (eps = 0): each particle moves
    uniformly on a circle, so its snap is -omega^2 times its acceleration."""
    m = np.array([0.5, 0.5])
    d = 1.3
    w = math.sqrt(1.0 / d ** 3)  # G (m1 + m2) / d^3
    r = np.array([[d / 2, 0.0, 0.0], [-d / 2, 0.0, 0.0]])
    v = np.array([[0.0, w * d / 2, 0.0], [0.0, -w * d / 2, 0.0]])
    a_true = orc.force(m, r, v, 0.0)[0]
    a, j, s, _ = orc.force_snap(m, r, v, a_true, 0.0)
    assert np.allclose(s, -w * w * a, rtol=0, atol=1e-14 * np.abs(s).max())
    assert np.allclose(j, -w * w * v / 2 * 0 + np.cross([0, 0, w], a), atol=1e-14)


def _poly(coef, t, k):
    """k-th derivative of sum_p coef[p] t^p / p! (vector coefficients)."""
    out = np.zeros(3)
    for p in range(k, len(coef)):
        out += coef[p] * t ** (p - k) / math.factorial(p - k)
    return out


@pytest.mark.parametrize("degree", [6, 7])
def test_corrector_exact_for_polynomial_trajectories(orc, degree):
    """x(t) a polynomial: with a = x'' of degree <= 5 the quintic interpolant
    is a itself, so v1, crackle, pop and the fifth derivative are exact; r1
    (a sixth-order quadrature of v) is exact while v has degree <= 5."""
    rng = np.random.default_rng(degree)
    coef = rng.normal(size=(degree + 1, 3))
    h = 0.37
    got = orc.hermite6_correct(*[_poly(coef, 0.0, k) for k in range(5)],
                               *[_poly(coef, h, k) for k in (2, 3, 4)], h)
    r1, v1, c1, d1, x1 = got
    assert np.allclose(v1, _poly(coef, h, 1), rtol=1e-13, atol=1e-13)
    for k, val in ((5, c1), (6, d1), (7, x1)):
        assert np.allclose(val, _poly(coef, h, k), rtol=1e-9, atol=1e-9)
    if degree == 6:
        assert np.allclose(r1, _poly(coef, h, 0), rtol=1e-13, atol=1e-13)
    else:
        assert not np.allclose(r1, _poly(coef, h, 0), rtol=1e-13, atol=1e-13)


def test_timestep_of_circular_motion(orc):
    """Every derivative of a uniformly rotating vector has |a^(k)| = w^k |a|,
    so the criterion gives eta / w, and it scales with time."""
    w, A, eta = 3.0, 2.0, 0.1
    ders = [A * w ** k * np.array([math.cos(k), math.sin(k), 0.0]) for k in range(6)]
    assert orc.aarseth6_dt(eta, *ders) == pytest.approx(eta / w, rel=1e-14)
    lam = 0.25  # t -> lam t: a^(k) -> a^(k) / lam^k, dt -> lam dt
    scaled = [d / lam ** k for k, d in enumerate(ders)]
    assert orc.aarseth6_dt(eta, *scaled) == pytest.approx(lam * eta / w, rel=1e-13)
    z = np.zeros(3)
    assert math.isinf(orc.aarseth6_dt(eta, ders[0], z, z, z, z, z))


def _kepler(e=0.5):
    m = np.array([0.5, 0.5])
    a_ax = 1.0
    rp = a_ax * (1 - e)
    vp = math.sqrt((1 + e) / rp)  # G (m1 + m2) = 1
    r = np.array([[rp / 2, 0, 0], [-rp / 2, 0, 0]])
    v = np.array([[0, vp / 2, 0], [0, -vp / 2, 0]])
    return m, r, v, 2 * math.pi * a_ax ** 1.5, -0.25 / (2 * a_ax)


def test_sixth_order_kepler_error_scales_as_eta_to_the_sixth(orc):
    """A Kepler orbit (e = 0.5, eps = 0) to t = 6 (just short of one period,
    2 pi), with dt_max = 1/4 so that the criterion, not the cap, sets the
    steps: halving eta doubles the block steps and divides the energy error
    by ~2^6 (measured 64-94 for eta 0.4 -> 0.05), where the fourth-order
    scheme of Sec. 2 divides it by ~2^4; and the sixth-order error at 227
    steps is below the fourth-order one at 641."""
    m, r, v, period, e_true = _kepler()
    t_end, dt_max = 6.0, 0.25
    runs = {}
    for eta in (0.2, 0.1):
        s = orc.State6(m, r, v, 0.0, eta, eta_start=eta / 16, dt_max=dt_max)
        assert abs(s.energy() - e_true) < 1e-14
        assert s.run(t_end) == orc.OK
        assert np.all(s.t == t_end)
        runs[eta] = (s.n_steps, abs(s.energy() - e_true) / abs(e_true))
    assert runs[0.1][0] == pytest.approx(2 * runs[0.2][0], rel=0.05)
    ratio = runs[0.2][1] / runs[0.1][1]
    assert 32 < ratio < 180, runs  # 2^6 = 64
    s4 = orc.State(m, r, v, 0.0, 0.025, eta_start=0.1 / 64, dt_max=dt_max)
    assert s4.run(t_end) == orc.OK
    assert s4.n_steps > 2 * runs[0.1][0]
    assert abs(s4.energy() - e_true) / abs(e_true) > 10 * runs[0.1][1]


def test_predictor_exact_for_a_quintic_trajectory(orc):
    """x(t) of degree 5: the Taylor predictor through crackle reproduces x,
    v = x' and a = x'' at any later time (reading H1)."""
    rng = np.random.default_rng(8)
    n = 4
    coefs = [rng.normal(size=(6, 3)) for _ in range(n)]
    t0 = np.array([0.0, 0.25, -0.5, 0.125])
    t = 0.75
    st = [np.array([_poly(c, tq, k) for c, tq in zip(coefs, t0)]) for k in range(6)]
    rp, vp, ap = orc.predict6(st[0], st[1], st[2], st[3], st[4], st[5], t0, t)
    for q in range(n):
        assert np.allclose(rp[q], _poly(coefs[q], t, 0), rtol=1e-13, atol=1e-13)
        assert np.allclose(vp[q], _poly(coefs[q], t, 1), rtol=1e-13, atol=1e-13)
        assert np.allclose(ap[q], _poly(coefs[q], t, 2), rtol=1e-13, atol=1e-13)
