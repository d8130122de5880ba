"""CUDA path (libnbody through its C ABI) against the FP64 oracle.

Tolerances:
  * FP64 force: per-particle relative error <= 1e-10 (double rounding of
    each pair, cancellation factors of a few hundred at most).
  * MIXED force: each pair is evaluated in FP32 (unit roundoff u = 2^-24),
    so |error_i| <= C u sum_j |term_ij| with C = 8 for acc and pot and 16 for
    jerk (derived from the operation count of a pair), and the median
    relative error stays at the FP32 level.
  * Scheduler (active list) and corrector: bit-exact (integer work, and a
    corrector written operation for operation in the equation order).
"""
import math
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
NTHREADS = os.cpu_count() or 1


def _rel(x, ref):
    x = np.atleast_2d(x.T).T if x.ndim == 1 else x
    ref = np.atleast_2d(ref.T).T if ref.ndim == 1 else ref
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _magnitude_sums(m, r, v, eps, idx, G=1.0):
    """sum_j |a_ij|, sum_j |j_ij|, sum_j |phi_ij| for the listed i (numpy)."""
    sa, sj, sp = [], [], []
    for i in idx:
        d = r - r[i]
        dv = v - v[i]
        r2 = (d * d).sum(1) + eps * eps
        r2[i] = np.inf
        rt = np.sqrt(r2)
        g = G * m / (r2 * rt)
        rv = (d * dv).sum(1)
        jt = g[:, None] * (dv - 3 * (rv / r2)[:, None] * d)
        sa.append((g * np.sqrt((d * d).sum(1))).sum())
        sj.append(np.linalg.norm(jt, axis=1).sum())
        sp.append((G * m / rt).sum())
    return np.array(sa), np.array(sj), np.array(sp)


def _state_at_rest(n, m, r, v):
    z = np.zeros((n, 3))
    return dict(m=m, r=r, v=v, a=z, j=z, t=np.zeros(n), dt=np.full(n, 1.0 / 16))


def _force_ctx(gpu, prec, m, r, v, eps):
    ctx = gpu.Context(prec)
    n = len(m)
    ctx.set_state(**_state_at_rest(n, m, r, v), eps=eps, eta=0.02)
    ctx.predict(0.0)
    return ctx


@pytest.mark.parametrize("n,n_act", [(1, 1), (63, 63), (64, 5), (1000, 1000), (1000, 37),
                                     (3001, 3001)])
def test_force_fp64_matches_oracle(gpu, orc, n, n_act):
    m, r, v = ics.plummer(n, 100 + n)
    eps = 4.0 / n if n > 1 else 0.1
    idx = ics.permutation(n, 7)[:n_act].astype(np.int32)
    with _force_ctx(gpu, "fp64", m, r, v, eps) as ctx:
        acc, jerk, pot = ctx.force(idx)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    if n == 1:
        assert np.all(acc == 0) and np.all(jerk == 0) and pot[0] == 0
        return
    assert np.max(_rel(acc, a0)) < 1e-10
    assert np.max(_rel(jerk, j0)) < 1e-10
    assert np.max(np.abs(pot - p0) / np.abs(p0)) < 1e-12


@pytest.mark.parametrize("n,n_act,eps", [(64, 64, 1 / 64), (1000, 1000, 4 / 1000),
                                         (1000, 37, 4 / 1000), (3001, 129, 0.0),
                                         (4096, 4096, 4 / 4096)])
def test_force_mixed_within_fp32_bound(gpu, orc, n, n_act, eps):
    m, r, v = ics.plummer(n, 200 + n)
    idx = ics.permutation(n, 8)[:n_act].astype(np.int32)
    with _force_ctx(gpu, "mixed", m, r, v, eps) as ctx:
        acc, jerk, pot = ctx.force(idx)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    sa, sj, sp = _magnitude_sums(m, r, v, eps, idx)
    ea = np.linalg.norm(acc - a0, axis=1)
    ej = np.linalg.norm(jerk - j0, axis=1)
    ep = np.abs(pot - p0)
    assert np.all(ea <= 8 * U32 * sa)
    assert np.all(ej <= 16 * U32 * sj)
    assert np.all(ep <= 8 * U32 * sp)
    assert np.median(_rel(acc, a0)) < 3e-7
    assert np.median(_rel(jerk, j0)) < 1e-6


@pytest.mark.parametrize("n,n_act,eps", [(64, 64, 1 / 64), (1000, 1000, 4 / 1000),
                                         (1000, 37, 4 / 1000), (3001, 129, 0.0),
                                         (4096, 4096, 4 / 4096)])
def test_force_ds_within_1e6_per_particle(gpu, orc, n, n_act, eps):
    """Double-single pair arithmetic: every particle within 1e-6 relative
    (the 1e-6 gate); the arithmetic carries ~44 bits, so the actual
    errors sit near 1e-11 even for particles whose forces nearly cancel."""
    m, r, v = ics.plummer(n, 200 + n)
    idx = ics.permutation(n, 8)[:n_act].astype(np.int32)
    with _force_ctx(gpu, "ds", m, r, v, eps) as ctx:
        acc, jerk, pot = ctx.force(idx)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    ra, rj = _rel(acc, a0), _rel(jerk, j0)
    rp = np.abs(pot - p0) / np.abs(p0)
    assert ra.max() < 1e-6 and rj.max() < 1e-6 and rp.max() < 1e-6
    sa, sj, sp = _magnitude_sums(m, r, v, eps, idx)
    # relative to the conditioning of each sum, DS is ~2^-40 accurate
    assert np.all(np.linalg.norm(acc - a0, axis=1) <= 1e-10 * sa)
    assert np.all(np.linalg.norm(jerk - j0, axis=1) <= 1e-10 * sj)


@pytest.mark.parametrize("split", [2, 4, 8])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "ds", "hybrid"])
@pytest.mark.parametrize("n,n_act,eps", [(1000, 37, 4 / 1000), (3001, 3001, 4 / 3001),
                                         (3001, 129, 0.0), (64, 5, 1 / 64)])
def test_force_j_split_within_warp(gpu, orc, prec, split, n, n_act, eps):
    """The j split inside a warp: `split` lanes share each i, lane slice s
    taking tile slots s, s + split, ...; the slices' partial sums are added by
    warp shuffles before the split-group tree.  Same bounds as the unsplit
    kernel (every group size, ragged blocks, the self pair at eps = 0)."""
    m, r, v = ics.plummer(n, 500 + n)
    idx = ics.permutation(n, 9)[:n_act].astype(np.int32)
    z = np.zeros((n, 3))
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    if prec == "hybrid":  # its near test reads the particles' own a, j
        aa, jj, _ = orc.force(m, r, v, eps, nthreads=NTHREADS)
    else:
        aa, jj = z, z
    with gpu.Context(prec, j_split=split) as ctx:
        ctx.set_state(m, r, v, aa, jj, np.zeros(n), np.full(n, 1.0 / 16), eps=eps, eta=0.02)
        ctx.predict(0.0)
        acc, jerk, pot = ctx.force(idx)
    sa, sj, sp = _magnitude_sums(m, r, v, eps, idx)
    ea = np.linalg.norm(acc - a0, axis=1)
    ej = np.linalg.norm(jerk - j0, axis=1)
    ep = np.abs(pot - p0)
    if prec == "fp64":
        assert _rel(acc, a0).max() < 1e-10 and _rel(jerk, j0).max() < 1e-10
    elif prec == "ds":
        assert np.all(ea <= 1e-10 * sa) and np.all(ej <= 1e-10 * sj)
    elif prec == "hybrid":
        assert _rel(acc, a0).max() < 1e-6 and _rel(jerk, j0).max() < 1e-6
        assert (ep / np.abs(p0)).max() < 1e-6
    else:
        assert np.all(ea <= 8 * U32 * sa) and np.all(ej <= 16 * U32 * sj)
        assert np.all(ep <= 8 * U32 * sp)


def test_force_j_split_rejects_bad_values(gpu):
    for bad in (3, 16, -1):
        with pytest.raises(gpu.NbError):
            gpu.Context("hybrid", j_split=bad)
    with pytest.raises(gpu.NbError):  # two i per lane has no j split
        gpu.Context("mixed", j_split=4, i_per_thread=2)


def test_force_self_exclusion_coincident_particles(gpu, orc):
    """Two particles at one point (eps > 0) still attract; the self pair does not."""
    m = np.array([0.3, 0.5, 0.2])
    r = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [1.0, -0.5, 0.25]])
    v = np.array([[0.0, 0.1, 0.0], [0.2, 0.0, 0.0], [0.0, 0.0, -0.3]])
    eps = 0.05
    a0, j0, p0 = orc.force(m, r, v, eps)
    for prec, tol in (("fp64", 1e-13), ("mixed", 1e-6), ("ds", 1e-10)):
        with _force_ctx(gpu, prec, m, r, v, eps) as ctx:
            acc, jerk, pot = ctx.force(np.arange(3, dtype=np.int32))
        np.testing.assert_allclose(acc, a0, rtol=tol, atol=tol * np.abs(a0).max())
        np.testing.assert_allclose(jerk, j0, rtol=tol, atol=tol * np.abs(j0).max())
        np.testing.assert_allclose(pot, p0, rtol=tol)


def test_force_after_prediction(gpu, orc):
    """nb_predict (Eqs. xpred, vpred) then nb_force against oracle predict + force."""
    n = 777
    m, r, v = ics.plummer(n, 9)
    rng = np.random.default_rng(1)
    a = rng.normal(0, 1, (n, 3))
    j = rng.normal(0, 5, (n, 3))
    dt = 2.0 ** -rng.integers(5, 9, n)
    t = np.zeros(n)
    eps = 0.01
    tp = 1.0 / 64
    rp, vp = orc.predict(r, v, a, j, t, tp)
    a0, j0, p0 = orc.force(m, rp, vp, eps, nthreads=NTHREADS)
    with gpu.Context("fp64") as ctx:
        ctx.set_state(m, r, v, a, j, t, dt, eps=eps, eta=0.02)
        ctx.predict(tp)
        acc, jerk, pot = ctx.force(np.arange(n, dtype=np.int32))
    assert np.max(_rel(acc, a0)) < 1e-10
    assert np.max(_rel(jerk, j0)) < 1e-10


@pytest.mark.parametrize("prec", ["ds", "hybrid", "mixed"])
def test_force_after_prediction_double_single_layout(gpu, orc, prec):
    """The predictor of the FP32-pipe precisions works in double-single from the
    FP64 state; the forces at the predicted positions must still meet each
    precision's bound against oracle predict + force (FP64 throughout)."""
    n = 1500
    m, r, v = ics.plummer(n, 19)
    rng = np.random.default_rng(3)
    eps = 4.0 / n
    # the particles' own a, j (HYBRID's near test reads them from the state);
    # zero and tiny components take the exact paths of the split
    a, j, _ = orc.force(m, r, v, eps, nthreads=NTHREADS)
    a[::97] = 0.0
    j[::11, 1] = 1e-30
    dt = 2.0 ** -rng.integers(5, 9, n)
    t = np.where(rng.uniform(size=n) < 0.5, 0.0, 1.0 / 64 - dt / 4)
    tp = 1.0 / 64
    idx = np.arange(n, dtype=np.int32)
    rp, vp = orc.predict(r, v, a, j, t, tp)
    a0, j0, p0 = orc.force(m, rp, vp, eps, nthreads=NTHREADS)
    sa, sj, sp = _magnitude_sums(m, rp, vp, eps, idx)
    with gpu.Context(prec) as ctx:
        ctx.set_state(m, r, v, a, j, t, dt, eps=eps, eta=0.02)
        ctx.predict(tp)
        acc, jerk, pot = ctx.force(idx)
    ea = np.linalg.norm(acc - a0, axis=1)
    ej = np.linalg.norm(jerk - j0, axis=1)
    ep = np.abs(pot - p0)
    if prec == "ds":
        assert np.all(ea <= 1e-10 * sa) and np.all(ej <= 1e-10 * sj)
        assert np.all(ep <= 1e-10 * sp)
    elif prec == "hybrid":
        assert _rel(acc, a0).max() < 1e-6 and _rel(jerk, j0).max() < 1e-6
        assert (ep / np.abs(p0)).max() < 1e-6
    else:
        assert np.all(ea <= 8 * U32 * sa) and np.all(ej <= 16 * U32 * sj)
        assert np.all(ep <= 8 * U32 * sp)


def _random_block_state(n, seed, T):
    """State with dyadic t, dt where a known subset is due at time T."""
    rng = np.random.default_rng(seed)
    m, r, v = ics.plummer(n, seed)
    a = rng.normal(0, 1, (n, 3))
    j = rng.normal(0, 3, (n, 3))
    lv = rng.integers(4, 9, n)
    dt = 2.0 ** -lv
    # particles due at T have t = T - dt; others are ahead of T
    due = rng.uniform(size=n) < 0.3
    t = np.where(due, T - dt, T)
    return m, r, v, a, j, t, dt, due


def test_select_matches_oracle_bit_exact(gpu, orc):
    # one-CTA select up to 32768 particles (edges at one tile, the limit),
    # the multi-block select above
    for n, seed in ((1, 1), (100, 2), (1024, 5), (1025, 6), (2048, 3), (5000, 4),
                    (32768, 7), (32769, 8), (70001, 9)):
        rng = np.random.default_rng(seed)
        m, r, v = ics.plummer(n, seed)
        dt = 2.0 ** -rng.integers(4, 12, n)
        t = dt * rng.integers(0, 8, n)
        z = np.zeros((n, 3))
        with gpu.Context("mixed") as ctx:
            ctx.set_state(m, r, v, z, z, t, dt, eps=0.01, eta=0.02)
            tn, idx = ctx.select()
            tn2, idx2 = ctx.select(t_end=-1.0)
        tref, iref = orc.select(t, dt)
        assert tn == tref
        assert np.array_equal(idx, iref)
        assert len(idx2) == 0


def test_correct_bit_exact_against_oracle(gpu, orc):
    n, T = 3000, 0.5
    m, r, v, a, j, t, dt, due = _random_block_state(n, 5, T)
    idx = np.nonzero(due)[0].astype(np.int32)
    rng = np.random.default_rng(6)
    a1 = a[idx] + rng.normal(0, 1e-3, (len(idx), 3))
    j1 = j[idx] + rng.normal(0, 1e-2, (len(idx), 3))
    with gpu.Context("fp64", dt_max=1.0 / 16) as ctx:
        ctx.set_state(m, r, v, a, j, t, dt, eps=0.01, eta=0.02)
        ctx.correct(T, idx, a1, j1)
        out = ctx.get_state()
    rp, vp = orc.predict(r[idx], v[idx], a[idx], j[idx], t[idx], T)
    for k, i in enumerate(idx):
        r1, v1, s0, c0 = orc.hermite_correct(rp[k], vp[k], a[i], j[i], a1[k], j1[k], dt[i])
        assert np.array_equal(out["r"][i], r1), (k, out["r"][i] - r1)
        assert np.array_equal(out["v"][i], v1)
        assert np.array_equal(out["a"][i], a1[k]) and np.array_equal(out["j"][i], j1[k])
        assert out["t"][i] == T
        dta = orc.aarseth_dt(0.02, a1[k], j1[k], s0 + c0 * dt[i], c0)
        st, dtn = orc.quantize_dt(dt[i], dta, T, 1.0 / 16)
        assert out["dt"][i] == dtn
    rest = np.nonzero(~due)[0]
    assert np.array_equal(out["r"][rest], r[rest]) and np.array_equal(out["t"][rest], t[rest])


@pytest.mark.parametrize("rel", [0.0, 2.0 ** -45, -(2.0 ** -45), 1e-7, -1e-7, 4e-6, -4e-6,
                                 3e-5, -3e-5, 0.3])
def test_correct_timestep_at_power_of_two_boundaries(gpu, orc, rel):
    """eta is set so that one particle's Eq. timestep value lands on, or a
    hair to either side of, its current step h (a power of two): the
    power-of-two rule must pick the oracle's step on both sides, whichever
    precision the kernel evaluates the formula in."""
    n, T = 400, 0.5
    m, r, v, a, j, t, dt, due = _random_block_state(n, 21, T)
    idx = np.nonzero(due)[0].astype(np.int32)
    rng = np.random.default_rng(22)
    a1 = a[idx] + rng.normal(0, 1e-3, (len(idx), 3))
    j1 = j[idx] + rng.normal(0, 1e-2, (len(idx), 3))
    rp, vp = orc.predict(r[idx], v[idx], a[idx], j[idx], t[idx], T)
    sc = []
    for k, i in enumerate(idx):
        _, _, s0, c0 = orc.hermite_correct(rp[k], vp[k], a[i], j[i], a1[k], j1[k], dt[i])
        sc.append((s0 + c0 * dt[i], c0))
    i0 = idx[0]
    unit = orc.aarseth_dt(1.0, a1[0], j1[0], *sc[0])
    eta = dt[i0] / unit * (1.0 + rel)
    with gpu.Context("fp64", dt_max=1.0 / 16) as ctx:
        ctx.set_state(m, r, v, a, j, t, dt, eps=0.01, eta=eta)
        ctx.correct(T, idx, a1, j1)
        out = ctx.get_state()
    for k, i in enumerate(idx):
        dta = orc.aarseth_dt(eta, a1[k], j1[k], *sc[k])
        _, dtn = orc.quantize_dt(dt[i], dta, T, 1.0 / 16)
        assert out["dt"][i] == dtn, (k, dta / dt[i])


def test_correct_rejects_particle_not_due(gpu):
    n, T = 100, 0.5
    m, r, v, a, j, t, dt, due = _random_block_state(n, 7, T)
    idx = np.nonzero(~due)[0][:3].astype(np.int32)
    with gpu.Context("fp64") as ctx:
        ctx.set_state(m, r, v, a, j, t, dt, eps=0.01, eta=0.02)
        with pytest.raises(gpu.NbError) as e:
            ctx.correct(T, idx, a[idx], j[idx])
        assert e.value.status == gpu.NB_ESTATE


def test_set_particles_matches_oracle_init(gpu, orc):
    n = 1000
    m, r, v = ics.plummer(n, 1)
    eps = 1.0 / 64
    s = orc.State(m, r, v, eps, 0.02, nthreads=NTHREADS)
    with gpu.Context("fp64") as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        out = ctx.get_state()
    assert np.max(_rel(out["a"], s.a)) < 1e-10
    assert np.max(_rel(out["j"], s.j)) < 1e-10
    assert np.array_equal(out["t"], s.t)
    assert np.mean(out["dt"] == s.dt) > 0.999


def test_block_step_equals_manual_sequence(gpu):
    """nb_block_step = nb_select + nb_predict + nb_force + nb_correct, bit for bit."""
    n = 2000
    m, r, v = ics.plummer(n, 12)
    with gpu.Context("mixed") as c1, gpu.Context("mixed") as c2:
        c1.set_particles(m, r, v, 4.0 / n, 0.02)
        c2.set_particles(m, r, v, 4.0 / n, 0.02)
        for _ in range(5):
            c1.block_step(1.0)
            tn, idx = c2.select(1.0)
            c2.predict(tn)
            c2.force(idx)
            c2.correct(tn, idx)
        s1, s2 = c1.get_state(), c2.get_state()
    for k in s1:
        assert np.array_equal(s1[k], s2[k]), k


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ds", "hybrid"])
def test_autotune_picks_valid_shapes_and_keeps_results(gpu, orc, prec):
    n = 3000
    m, r, v = ics.plummer(n, 31)
    eps = 4.0 / n
    idx = np.arange(n, dtype=np.int32)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    with gpu.Context(prec, autotune=True) as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)  # tunes on load
        tun = ctx.autotune()
        for b in ("small", "large"):
            assert tun[f"{b}_i_per_thread"] in (1, 2)
            assert 1 <= tun[f"{b}_ctas_per_sm"] <= 8
            assert tun[f"{b}_us"] > 0
        ctx.set_state(**_state_at_rest(n, m, r, v), eps=eps, eta=0.02)
        ctx.predict(0.0)
        for k in (17, 100, n):  # one block in each bucket
            acc, jerk, pot = ctx.force(idx[:k])
            if prec == "mixed":
                sa, sj, _ = _magnitude_sums(m, r, v, eps, idx[:k])
                assert np.all(np.linalg.norm(acc - a0[:k], axis=1) <= 8 * U32 * sa)
            else:
                tol = 1e-10 if prec == "fp64" else 1e-6
                assert np.max(_rel(acc, a0[:k])) < tol and np.max(_rel(jerk, j0[:k])) < tol
        ctx.set_particles(m, r, v, eps, 0.02)
        steps, inter = ctx.step_until(1.0 / 32)  # both launch variants in the graph
        assert steps > 0 and inter > 0


def test_errors_are_reported(gpu):
    m = np.array([1.0, 1.0])
    r = np.zeros((2, 3))
    v = np.zeros((2, 3))
    with gpu.Context("mixed") as ctx:
        with pytest.raises(gpu.NbError) as e:
            ctx.set_particles(m, r, v, 0.0, 0.02)  # eps = 0, coincident
        assert e.value.status == gpu.NB_ENONFINITE
        m, r, v = ics.plummer(10, 1)
        ctx.set_particles(m, r, v, 0.1, 0.02)  # reload clears the error
        with pytest.raises(gpu.NbError) as e:
            ctx.force(np.array([0, 10], dtype=np.int32))
        assert e.value.status == gpu.NB_EINVAL
        ctx.force(np.array([0, 9], dtype=np.int32))  # EINVAL is not sticky


def _energy(orc_state):
    return orc_state.energy()


def test_integration_fp64_plummer_n1024(gpu, orc):
    """Plummer N = 1024, eps = 1/64, eta = 0.02 to t = 0.5: energy drift of
    the FP64 GPU path within 2x the oracle's, and the same trajectory."""
    n, eps, eta, t_end = 1024, 1.0 / 64, 0.02, 0.5
    m, r, v = ics.plummer(n, 1)
    s = orc.State(m, r, v, eps, eta, nthreads=NTHREADS)
    E0 = s.energy()
    assert s.run(t_end) == 0
    dE_orc = abs(s.energy() - E0) / abs(E0)
    with gpu.Context("fp64") as ctx:
        ctx.set_particles(m, r, v, eps, eta)
        K0, W0 = ctx.energy()
        assert (K0 + W0) == pytest.approx(E0, rel=1e-12)
        steps, inter = ctx.step_until(t_end)
        K1, W1 = ctx.energy()
        out = ctx.get_state()
    dE_gpu = abs(K1 + W1 - E0) / abs(E0)
    assert np.all(out["t"] == t_end)
    assert dE_gpu <= 2 * dE_orc + 1e-12
    assert steps == pytest.approx(s.n_steps, rel=0.02)
    assert inter == pytest.approx(s.n_inter, rel=0.02)
    assert np.max(np.abs(out["r"] - s.r)) < 1e-6


def test_integration_mixed_plummer_n1024(gpu, orc):
    n, eps, eta, t_end = 1024, 1.0 / 64, 0.02, 0.5
    m, r, v = ics.plummer(n, 1)
    s = orc.State(m, r, v, eps, eta, nthreads=NTHREADS)
    E0 = s.energy()
    assert s.run(t_end) == 0
    dE_orc = abs(s.energy() - E0) / abs(E0)
    with gpu.Context("mixed") as ctx:
        ctx.set_particles(m, r, v, eps, eta)
        ctx.step_until(t_end)
        K1, W1 = ctx.energy(fp64_potential=True)
    dE_gpu = abs(K1 + W1 - E0) / abs(E0)
    # the paper's mixed scheme floors near 1e-9 relative energy error
    assert dE_gpu <= 2 * dE_orc + 2e-9
