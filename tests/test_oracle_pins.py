"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test fixes one piece of Sec. 2 of the paper to mathematics or physics
that is independent of how the oracle writes its formulas: derivatives of
the potential, Taylor's theorem, exactness of the Hermite interpolation on
polynomials, Newton's third law, a ring's closed-form field, Kepler orbits.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _random_system(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5, 2.0, n) / n
    r = rng.normal(0, spread, (n, 3))
    v = rng.normal(0, 0.5, (n, 3))
    return m, r, v


# --- Eqs. acc, jrk, pot --------------------------------------------------------
def test_force_matches_symbolic_derivatives_of_potential(orc):
    """a_i = -grad_i phi_i and j_i = d a_i/dt, differentiated symbolically.

    phi is written once as the softened potential sum (Eq. pot); sympy
    differentiates it, so a dropped term, a wrong sign or exponent in the
    oracle's acc/jerk expressions (Eqs. acc, jrk) cannot match by accident.
    Integer-valued coordinates, evaluated at 40 digits.
    """
    sympy = pytest.importorskip("sympy")
    pos = [(0, 0, 0), (3, 1, -2), (-1, 4, 2), (2, -3, 1), (-2, -1, -3)]
    vel = [(1, 0, -1), (0, 2, 1), (-1, -1, 0), (2, 1, 3), (0, -2, 1)]
    mass = [1, 2, 3, 1, 2]
    G, eps = sympy.Rational(7, 5), sympy.Rational(1, 2)
    t = sympy.Symbol("t")
    n = len(pos)
    R = [[pos[k][d] + vel[k][d] * t for d in range(3)] for k in range(n)]
    m = np.array(mass, float)
    r = np.array(pos, float)
    v = np.array(vel, float)
    acc, jerk, pot = orc.force(m, r, v, float(eps), float(G))
    for i in range(n):
        xs = sympy.symbols("x y z")
        phi = 0
        for j in range(n):
            if j == i:
                continue
            d2 = sum((R[j][d] - xs[d]) ** 2 for d in range(3)) + eps ** 2
            phi += -G * mass[j] / sympy.sqrt(d2)
        a_sym = [-sympy.diff(phi, xs[d]) for d in range(3)]
        a_t = [a.subs({xs[d]: R[i][d] for d in range(3)}) for a in a_sym]
        j_t = [sympy.diff(a, t) for a in a_t]
        for d in range(3):
            a_ref = float(sympy.N(a_t[d].subs(t, 0), 40))
            j_ref = float(sympy.N(j_t[d].subs(t, 0), 40))
            assert acc[i, d] == pytest.approx(a_ref, rel=1e-13, abs=1e-15)
            assert jerk[i, d] == pytest.approx(j_ref, rel=1e-13, abs=1e-15)
        p_ref = float(sympy.N(phi.subs({xs[d]: R[i][d] for d in range(3)}).subs(t, 0), 40))
        assert pot[i] == pytest.approx(p_ref, rel=1e-14)


def test_acc_is_minus_gradient_of_potential_finite_difference(orc):
    """Central differences of phi_i(r_i) reproduce -a_i to O(h^2)."""
    m, r, v = _random_system(12, 1)
    eps = 0.05
    acc, _, _ = orc.force(m, r, v, eps)
    h = 1e-5
    for i in (0, 5, 11):
        g = np.zeros(3)
        for d in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, d] += h
            rm[i, d] -= h
            _, _, pp = orc.force(m, rp, v, eps, idx=[i])
            _, _, pm = orc.force(m, rm, v, eps, idx=[i])
            g[d] = (pp[0] - pm[0]) / (2 * h)
        np.testing.assert_allclose(-g, acc[i], rtol=1e-7, atol=1e-9)


def test_jerk_is_time_derivative_of_acc_along_drift(orc):
    """[a(r + h v) - a(r - h v)] / 2h -> j with error O(h^2)."""
    m, r, v = _random_system(20, 2)
    eps = 0.02
    _, jerk, _ = orc.force(m, r, v, eps)
    errs = []
    for h in (2e-4, 1e-4):
        ap, _, _ = orc.force(m, r + h * v, v, eps)
        am, _, _ = orc.force(m, r - h * v, v, eps)
        fd = (ap - am) / (2 * h)
        errs.append(np.max(np.abs(fd - jerk)) / np.max(np.abs(jerk)))
    assert errs[1] < 1e-6
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0  # second order: halving h quarters the error


def test_ring_closed_form_on_axis(orc):
    """K equal masses on a ring of radius R: on-axis softened field is exact.

    phi(z) = -G M / sqrt(R^2 + z^2 + eps^2),
    a_z = -G M z / (R^2 + z^2 + eps^2)^(3/2), a_x = a_y = 0.
    """
    K, R, z, M, eps, G = 12, 1.3, 0.7, 2.5, 0.1, 0.9
    ang = 2 * np.pi * np.arange(K) / K
    r = np.zeros((K + 1, 3))
    r[:K, 0] = R * np.cos(ang)
    r[:K, 1] = R * np.sin(ang)
    r[K] = (0.0, 0.0, z)
    m = np.full(K + 1, M / K)
    m[K] = 1.0
    v = np.zeros((K + 1, 3))
    acc, jerk, pot = orc.force(m, r, v, eps, G, idx=[K])
    s2 = R * R + z * z + eps * eps
    assert pot[0] == pytest.approx(-G * M / math.sqrt(s2), rel=1e-14)
    assert acc[0, 2] == pytest.approx(-G * M * z / s2 ** 1.5, rel=1e-14)
    assert abs(acc[0, 0]) < 1e-14 and abs(acc[0, 1]) < 1e-14
    np.testing.assert_allclose(jerk[0], 0.0, atol=1e-14)


def test_newton_third_law_momentum_and_angular_momentum(orc):
    """sum m a = 0, sum m j = 0 and sum m r x a = 0 for a full evaluation."""
    m, r, v = _random_system(64, 3)
    acc, jerk, _ = orc.force(m, r, v, 0.01)
    scale_a = np.sum(m[:, None] * np.abs(acc))
    scale_j = np.sum(m[:, None] * np.abs(jerk))
    assert np.max(np.abs((m[:, None] * acc).sum(0))) < 1e-14 * scale_a
    assert np.max(np.abs((m[:, None] * jerk).sum(0))) < 1e-14 * scale_j
    torque = (m[:, None] * np.cross(r, acc)).sum(0)
    assert np.max(np.abs(torque)) < 1e-13 * scale_a


def test_self_pair_excluded_by_index_not_distance(orc):
    """Two distinct particles at one point with eps > 0 still interact."""
    m = np.array([1.0, 2.0, 3.0])
    r = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    v = np.zeros((3, 3))
    eps = 0.5
    _, _, pot = orc.force(m, r, v, eps)
    assert pot[0] == pytest.approx(-2.0 / eps - 3.0 / math.sqrt(1 + eps * eps), rel=1e-15)


def test_self_term_alone_gives_zero(orc):
    m, r, v = np.array([1.0]), np.zeros((1, 3)), np.ones((1, 3))
    acc, jerk, pot = orc.force(m, r, v, 0.0)
    assert np.all(acc == 0) and np.all(jerk == 0) and pot[0] == 0


# --- Eqs. xpred, vpred ---------------------------------------------------------
def test_predictor_is_exact_for_cubic_trajectories(orc):
    """Taylor's theorem: a cubic path is reproduced by its first 4 derivatives."""
    rng = np.random.default_rng(4)
    n = 50
    c = rng.normal(size=(4, n, 3))  # x(t) = c0 + c1 t + c2 t^2 + c3 t^3
    t0 = rng.uniform(0, 1, n)
    t = 1.375

    def deriv(tau, k):
        tau = tau[:, None]
        if k == 0:
            return c[0] + c[1] * tau + c[2] * tau ** 2 + c[3] * tau ** 3
        if k == 1:
            return c[1] + 2 * c[2] * tau + 3 * c[3] * tau ** 2
        if k == 2:
            return 2 * c[2] + 6 * c[3] * tau
        return 6 * c[3] + 0 * tau

    rp, vp = orc.predict(deriv(t0, 0), deriv(t0, 1), deriv(t0, 2), deriv(t0, 3), t0, t)
    tt = np.full(n, t)
    np.testing.assert_allclose(rp, deriv(tt, 0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(vp, deriv(tt, 1), rtol=1e-12, atol=1e-12)


# --- Sec. 2 Hermite interpolation and corrector --------------------------------
def test_hermite_snap_crackle_exact_for_cubic_acceleration(orc):
    """If a(t) is a cubic, s0 = a''(0) and c0 = a'''(0) exactly."""
    rng = np.random.default_rng(5)
    q = rng.normal(size=(4, 3))  # a(t) = q0 + q1 t + q2 t^2 + q3 t^3
    h = 0.125
    a0, j0 = q[0], q[1]
    a1 = q[0] + q[1] * h + q[2] * h ** 2 + q[3] * h ** 3
    j1 = q[1] + 2 * q[2] * h + 3 * q[3] * h ** 2
    _, _, s0, c0 = orc.hermite_correct(np.zeros(3), np.zeros(3), a0, j0, a1, j1, h)
    np.testing.assert_allclose(s0, 2 * q[2], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c0, 6 * q[3], rtol=1e-12, atol=1e-12)


def test_predictor_corrector_exact_for_quintic_trajectory(orc):
    """A quintic path has a cubic acceleration: predict + correct is exact.

    This pins every coefficient of the corrector (1/24, 1/120, 1/6, 1/24)."""
    rng = np.random.default_rng(6)
    c = rng.normal(size=(6, 3))
    h = 0.0625

    def x(t, k):
        out = np.zeros(3)
        for p in range(k, 6):
            out += c[p] * math.factorial(p) / math.factorial(p - k) * t ** (p - k)
        return out

    rp, vp = orc.predict(x(0, 0)[None], x(0, 1)[None], x(0, 2)[None], x(0, 3)[None], [0.0], h)
    r1, v1, _, _ = orc.hermite_correct(rp[0], vp[0], x(0, 2), x(0, 3), x(h, 2), x(h, 3), h)
    np.testing.assert_allclose(r1, x(h, 0), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(v1, x(h, 1), rtol=1e-13, atol=1e-14)


# --- Eq. timestep and the hierarchical rule -------------------------------------
def test_aarseth_circular_orbit(orc):
    """Uniform circular motion: |a|=w^2 R, |j|=w^3 R, |s|=w^4 R, |c|=w^5 R -> eta/w."""
    w, R, eta = 2.7, 0.8, 0.02
    ph = 0.3
    u = np.array([math.cos(ph), math.sin(ph), 0.0])
    t = np.array([-math.sin(ph), math.cos(ph), 0.0])
    a = -w ** 2 * R * u
    j = -w ** 3 * R * t
    s = w ** 4 * R * u
    c = w ** 5 * R * t
    assert orc.aarseth_dt(eta, a, j, s, c) == pytest.approx(eta / w, rel=1e-14)


def test_aarseth_time_rescaling(orc):
    """Stretching time by k (a -> a/k^2, j -> j/k^3, ...) stretches dt by k."""
    rng = np.random.default_rng(7)
    a, j, s, c = rng.normal(size=(4, 3))
    k = 3.0
    dt1 = orc.aarseth_dt(0.02, a, j, s, c)
    dt2 = orc.aarseth_dt(0.02, a / k ** 2, j / k ** 3, s / k ** 4, c / k ** 5)
    assert dt2 == pytest.approx(k * dt1, rel=1e-13)


def test_quantize_rules(orc):
    dmax = 1.0 / 16
    # shrink: halve until <= candidate
    st, dt = orc.quantize_dt(2 ** -6, 0.004, 2 ** -6 * 3, dmax)
    assert st == 0 and dt == 2 ** -8
    # keep: candidate between dt and 2 dt
    st, dt = orc.quantize_dt(2 ** -6, 1.5 * 2 ** -6, 2 ** -6 * 3, dmax)
    assert dt == 2 ** -6
    # grow only where t_next is a multiple of 2 dt
    st, dt = orc.quantize_dt(2 ** -6, 1.0, 2 ** -6 * 3, dmax)
    assert dt == 2 ** -6
    st, dt = orc.quantize_dt(2 ** -6, 1.0, 2 ** -6 * 4, dmax)
    assert dt == 2 ** -5
    # never above dt_max
    st, dt = orc.quantize_dt(dmax, 1.0, 1.0, dmax)
    assert dt == dmax
    # below dt_min is an error
    st, _ = orc.quantize_dt(2 ** -6, 1e-15, 2 ** -6, dmax, dt_min=2.0 ** -40)
    assert st == orc.EDTMIN


def test_initial_dt_power_of_two(orc):
    st, dt = orc.initial_dt(0.01, [1.0, 0, 0], [0, 3.0, 0], 1 / 16)
    assert st == 0 and dt == 2.0 ** math.floor(math.log2(0.01 / 3.0))
    st, dt = orc.initial_dt(0.01, [1.0, 0, 0], [0, 0, 0], 1 / 16)
    assert dt == 1 / 16


def test_isolated_particle_steps_at_dt_max(orc):
    """Reading R5: a particle that feels nothing (a = j = s = c = 0) has no
    timestep constraint; a one-particle system moves in a straight line."""
    z = np.zeros(3)
    assert orc.aarseth_dt(0.02, z, z, z, z) == float("inf")
    st, dt = orc.initial_dt(0.01, z, z, 1 / 16)
    assert st == 0 and dt == 1 / 16
    s = orc.State([1.0], [[0.5, 0.0, 0.0]], [[0.25, -1.0, 2.0]], 0.0, 0.02)
    assert s.run(1.0) == 0 and s.n_steps == 16
    np.testing.assert_allclose(s.r[0], [0.75, -1.0, 2.0], rtol=0, atol=1e-15)


def test_select_against_brute_force(orc):
    rng = np.random.default_rng(8)
    n = 500
    dt = 2.0 ** -rng.integers(4, 10, n)
    t = dt * rng.integers(0, 4, n)
    tn, idx = orc.select(t, dt)
    assert tn == np.min(t + dt)
    assert list(idx) == [i for i in range(n) if t[i] + dt[i] == tn]


# --- the integrator as a whole ---------------------------------------------------
def _kepler(e=0.5, a=1.0, m1=0.6, m2=0.4, G=1.0):
    """Two bodies at apocentre in their centre-of-mass frame."""
    M = m1 + m2
    ra = a * (1 + e)
    va = math.sqrt(G * M / a * (1 - e) / (1 + e))
    rel_r = np.array([ra, 0.0, 0.0])
    rel_v = np.array([0.0, va, 0.0])
    r = np.array([-m2 / M * rel_r, m1 / M * rel_r])
    v = np.array([-m2 / M * rel_v, m1 / M * rel_v])
    return np.array([m1, m2]), r, v


def test_kepler_energy_period_and_fourth_order(orc):
    """e = 0.5, eps = 0: energy -G m1 m2 / 2a, period 2 pi sqrt(a^3 / G M);
    the energy error falls as eta^4 (Sec. 4, n_step^-4 scaling)."""
    m, r, v = _kepler()
    E0 = -m[0] * m[1] / 2.0
    P = 2 * math.pi
    dt_max = 1.0 / 64
    t_end = math.floor(P / dt_max) * dt_max
    errs = []
    for eta in (0.04, 0.02):
        s = orc.State(m, r, v, 0.0, eta, dt_max=dt_max)
        assert s.energy() == pytest.approx(E0, rel=1e-14)
        assert s.run(t_end) == 0
        assert np.all(s.t == t_end)
        errs.append(abs(s.energy() - E0) / abs(E0))
        # t_end is P - delta with delta < dt_max: the pair is just short of
        # apocentre, at angle -omega_apo * delta and separation a (1 + e).
        rel = s.r[1] - s.r[0]
        delta = P - t_end
        omega_apo = math.sqrt(0.5 / 1.5) / 1.5
        assert math.atan2(rel[1], rel[0]) == pytest.approx(-omega_apo * delta, abs=1e-3)
        assert np.linalg.norm(rel) == pytest.approx(1.5, rel=1e-5)
    assert errs[1] < 1e-6
    ratio = errs[0] / errs[1]
    assert 8.0 < ratio < 32.0  # 2^4 = 16 for a fourth-order scheme


def test_block_scheduler_invariants(orc):
    from paper_1104_2700_gb300 import ics
    m, r, v = ics.plummer(128, 11)
    s = orc.State(m, r, v, 4.0 / 128, 0.02)
    for k in range(1, 5):
        t_sync = k / 16
        assert s.run(t_sync) == 0
        assert np.all(s.t == t_sync)
        lg = np.log2(s.dt)
        assert np.all(lg == np.round(lg)) and np.all(s.dt <= 1 / 16)
        assert np.all(np.fmod(s.t, s.dt) == 0)
