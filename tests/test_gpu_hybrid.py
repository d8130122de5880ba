"""Hybrid precision (NB_HYBRID) against the FP64 oracle.

Far pairs run in FP32 and near pairs (whose acceleration or jerk term could
exceed 10 % of the particle's own |a| or |j|) in double-single.  The near
test reads |a|, |j| from the state, so every test here loads the oracle's
a, j at t = 0 into the state first; with a = j = 0 every pair is near and
the result is the DS one.

Bar: every particle within 1e-6 relative in acc, jerk and pot (the north-
star bound).  The errors are FP32-level (median ~1e-8), which also shows
the FP32 far path ran.
"""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _ctx(gpu, prec, m, r, v, eps, a, j):
    n = len(m)
    ctx = gpu.Context(prec)
    ctx.set_state(m, r, v, a, j, np.zeros(n), np.full(n, 1.0 / 16), eps=eps, eta=0.02)
    ctx.predict(0.0)
    return ctx


@pytest.mark.parametrize("n,n_act,eps", [(64, 64, 1 / 64), (1000, 1000, 4 / 1000),
                                         (1000, 37, 4 / 1000), (3001, 129, 1e-3),
                                         (4096, 4096, 4 / 4096), (8191, 700, 4 / 8191)])
def test_force_hybrid_within_1e6_per_particle(gpu, orc, n, n_act, eps):
    m, r, v = ics.plummer(n, 500 + n)
    a_all, j_all, _ = orc.force(m, r, v, eps, nthreads=NTHREADS)
    idx = ics.permutation(n, 8)[:n_act].astype(np.int32)
    with _ctx(gpu, "hybrid", m, r, v, eps, a_all, j_all) as ctx:
        acc, jerk, pot = ctx.force(idx)
    a0, j0, p0 = a_all[idx], j_all[idx], orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)[2]
    ea, ej = _rel(acc, a0), _rel(jerk, j0)
    ep = np.abs(pot - p0) / np.abs(p0)
    assert max(ea.max(), ej.max(), ep.max()) < 1e-6
    if n >= 1000:
        # most pairs took the FP32 path: FP32-level, not DS-level, errors
        assert 1e-11 < np.median(ea) < 1e-7


def test_hybrid_without_estimates_is_double_single(gpu, orc):
    """With a = j = 0 in the state every pair is near: the DS result."""
    n, eps = 2000, 4 / 2000
    m, r, v = ics.plummer(n, 77)
    z = np.zeros((n, 3))
    idx = np.arange(0, n, 3, dtype=np.int32)
    with _ctx(gpu, "hybrid", m, r, v, eps, z, z) as ctx:
        ah, jh, ph = ctx.force(idx)
    with _ctx(gpu, "ds", m, r, v, eps, z, z) as ctx:
        ad, jd, pd = ctx.force(idx)
    assert np.max(_rel(ah, ad)) < 1e-12 and np.max(_rel(jh, jd)) < 1e-12
    assert np.max(np.abs(ph - pd) / np.abs(pd)) < 1e-12


def test_hybrid_near_pairs_rescue_cancellation(gpu, orc):
    """A particle between two heavy neighbours: its pair forces nearly
    cancel (|a| is ~1e-4 of the pair terms).  FP32 pair arithmetic cannot
    give 1e-6 there; the near test sends both pairs to DS."""
    n = 1500
    m, r, v = ics.plummer(n, 5)
    m = m.copy()
    r = r.copy()
    m[1] = m[2] = 50 * m[0]
    r[1] = r[0] + np.array([1e-2, 0.0, 0.0])
    r[2] = r[0] - np.array([1e-2, 1e-6, 0.0])
    eps = 1e-4
    a_all, j_all, _ = orc.force(m, r, v, eps, nthreads=NTHREADS)
    idx = np.array([0], dtype=np.int32)
    with _ctx(gpu, "hybrid", m, r, v, eps, a_all, j_all) as ctx:
        acc, jerk, pot = ctx.force(idx)
    assert _rel(acc, a_all[idx]).max() < 1e-6
    assert _rel(jerk, j_all[idx]).max() < 1e-6


@pytest.mark.parametrize("prec", ["hybrid", "ds"])
@pytest.mark.parametrize("t_end", [0.5, 1.0])
def test_integration_hybrid_plummer_n1024(gpu, orc, t_end, prec):
    """The N = 1024 workload (eps = 1/64, eta = 0.02) to t = 0.5 and t = 1:
    relative energy drift within 2x the oracle's, the bound stated for the
    reduced-precision path (only 1e-13 is added, the rounding of the FP64
    energy sums themselves), and no timestep collapse: the block steps stay
    within 5 % of the oracle's (MIXED takes ~200x more on this workload).
    DS, the other precision that integrates, is held to the same bounds."""
    n, eps, eta = 1024, 1.0 / 64, 0.02
    m, r, v = ics.plummer(n, 1)
    s = orc.State(m, r, v, eps, eta, nthreads=NTHREADS)
    E0 = s.energy()
    assert s.run(t_end) == 0
    dE_orc = abs(s.energy() - E0) / abs(E0)
    with gpu.Context(prec) as ctx:
        ctx.set_particles(m, r, v, eps, eta)
        steps, inter = ctx.step_until(t_end)
        K1, W1 = ctx.energy(fp64_potential=True)
    dE_gpu = abs(K1 + W1 - E0) / abs(E0)
    assert dE_gpu <= 2 * dE_orc + 1e-13, (dE_gpu, dE_orc)
    assert steps == pytest.approx(s.n_steps, rel=0.05)


def test_hybrid_integration_guard_prevents_step_collapse(gpu):
    """Member 8 of the ensemble workload (Plummer N = 7461, eps = 4/N) holds a
    particle with |a| = 0.045 and |j| = 39.  Its FP32 far field leaves
    ~1.5e-8 absolute noise in a (3e-7 relative, inside the force bound), but
    crackle divides a0 - a1 by dt^3, and without the integration guard its
    timestep collapsed from 2^-17 to 2^-23 (43556 block steps to t = 1/64
    against DS's 1292).  With the guard the schedules agree."""
    sizes, off, ms, rs, vs, eps = ics.ensemble(256, 4, 1000)
    q = 8
    lo, hi = off[q], off[q + 1]
    steps = {}
    for prec in ("ds", "hybrid"):
        with gpu.Context(prec) as ctx:
            ctx.set_particles(ms[lo:hi], rs[lo:hi], vs[lo:hi], float(eps[q]), 0.02)
            steps[prec], _ = ctx.step_until(1.0 / 64)
            dt = ctx.get_state()["dt"]
        if prec == "hybrid":
            assert dt.min() >= 2.0 ** -17
    assert steps["hybrid"] == pytest.approx(steps["ds"], rel=0.05)


@pytest.mark.parametrize("it", [1, 2])
def test_force_hybrid_launch_shapes_agree(gpu, orc, it):
    """One and two i particles per lane: both within 1e-6 everywhere."""
    n, eps = 5000, 4 / 5000
    m, r, v = ics.plummer(n, 606)
    a_all, j_all, p_all = orc.force(m, r, v, eps, nthreads=NTHREADS)
    idx = np.arange(n, dtype=np.int32)
    with gpu.Context("hybrid", i_per_thread=it) as ctx:
        ctx.set_state(m, r, v, a_all, j_all, np.zeros(n), np.full(n, 1.0 / 16), eps=eps, eta=0.02)
        ctx.predict(0.0)
        acc, jerk, pot = ctx.force(idx)
    assert max(_rel(acc, a_all).max(), _rel(jerk, j_all).max(),
               (np.abs(pot - p_all) / np.abs(p_all)).max()) < 1e-6
