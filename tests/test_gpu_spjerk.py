"""MIXED_SPJ: MIXED with the jerk summed in plain FP32 over each warp's run
of j, the accumulation of the paper's production kernel (Sec. 4, Fig.
err_snp_djerk), against the FP64 oracle and against MIXED.

Tolerances:
  * A plain FP32 sum of L terms errs by at most (L - 1) u sum |terms| to
    first order (u = 2^-24), on top of the rounding of each pair term, which
    the MIXED bound already covers with 16 u sum |terms|.  A run holds at most
    N terms, so |error_i| <= (16 + N) u sum_j |j_ij|.
  * Acceleration and potential take exactly MIXED's arithmetic, so under the
    same launch shape they agree with MIXED bit for bit.
"""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
NTHREADS = os.cpu_count() or 1


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _magnitude_sums(m, r, v, eps, idx):
    sa, sj, sp = [], [], []
    for i in idx:
        d = r - r[i]
        dv = v - v[i]
        r2 = (d * d).sum(1) + eps * eps
        r2[i] = np.inf
        rt = np.sqrt(r2)
        g = m / (r2 * rt)
        rv = (d * dv).sum(1)
        jt = g[:, None] * (dv - 3 * (rv / r2)[:, None] * d)
        sa.append((g * np.sqrt((d * d).sum(1))).sum())
        sj.append(np.linalg.norm(jt, axis=1).sum())
        sp.append((m / rt).sum())
    return np.array(sa), np.array(sj), np.array(sp)


def _forces(gpu, prec, m, r, v, eps, idx):
    n = len(m)
    z = np.zeros((n, 3))
    with gpu.Context(prec) as ctx:
        ctx.set_state(m, r, v, z, z, np.zeros(n), np.full(n, 1.0 / 16), eps, 0.02)
        ctx.predict(0.0)
        return ctx.force(idx)


@pytest.mark.parametrize("n,n_act,eps", [(64, 64, 1 / 64), (1000, 1000, 4 / 1000),
                                         (1000, 37, 4 / 1000), (3001, 129, 0.0),
                                         (8192, 8192, 4 / 8192)])
def test_spj_within_plain_sum_bound(gpu, orc, n, n_act, eps):
    m, r, v = ics.plummer(n, 300 + n)
    idx = ics.permutation(n, 12)[:n_act].astype(np.int32)
    acc, jerk, pot = _forces(gpu, "mixed_spj", m, r, v, eps, idx)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    sa, sj, sp = _magnitude_sums(m, r, v, eps, idx)
    assert np.all(np.linalg.norm(acc - a0, axis=1) <= 8 * U32 * sa)
    assert np.all(np.linalg.norm(jerk - j0, axis=1) <= (16 + n) * U32 * sj)
    assert np.all(np.abs(pot - p0) <= 8 * U32 * sp)


@pytest.mark.parametrize("n,n_act", [(4096, 4096), (4096, 129), (20000, 20000)])
def test_spj_acc_pot_identical_to_mixed(gpu, n, n_act):
    m, r, v = ics.plummer(n, 17)
    eps = 4.0 / n
    idx = ics.permutation(n, 13)[:n_act].astype(np.int32)
    a1, j1, p1 = _forces(gpu, "mixed", m, r, v, eps, idx)
    a2, j2, p2 = _forces(gpu, "mixed_spj", m, r, v, eps, idx)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    if n_act == n:
        # every warp sums many tiles of j: the plain FP32 jerk sum differs
        assert not np.array_equal(j1, j2)


def test_spj_jerk_error_exceeds_compensated_at_large_n(gpu):
    """Sec. 4: summing the jerk in SP makes its error grow with N.  At
    N = 16384 (every warp summing tens of tiles of j in one FP32 sum) the
    median jerk error against the FP64 path is several times MIXED's, whose
    per-tile partial sums are folded into compensated accumulators."""
    n = 16384
    m, r, v = ics.plummer(n, 11)
    eps = 4.0 / n
    idx = np.arange(n, dtype=np.int32)
    a0, j0, _ = _forces(gpu, "fp64", m, r, v, eps, idx)
    _, jm, _ = _forces(gpu, "mixed", m, r, v, eps, idx)
    _, js, _ = _forces(gpu, "mixed_spj", m, r, v, eps, idx)
    em, es = np.median(_rel(jm, j0)), np.median(_rel(js, j0))
    assert es > 2.0 * em


def test_mixed_accuracy_matches_fig_err_snp(gpu, orc):
    """MIXED (the paper's scheme on FP32 pipes) against Sec. 4's stated
    accuracy (tests/golden/paper_figures.json): on Plummer models with eps = 4/N
    and every particle active, median acceleration errors within a factor of
    10 of 1e-8, potentials no worse, jerks less accurate than accelerations."""
    import json
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "paper_figures.json")) as fh:
        typical = json.load(fh)["acc_pot_relative_error_typical"]["value"]
    for n in (1024, 4096):
        m, r, v = ics.plummer(n, 11)
        eps = 4.0 / n
        idx = np.arange(n, dtype=np.int32)
        acc, jerk, pot = _forces(gpu, "mixed", m, r, v, eps, idx)
        a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
        acc_med = np.median(_rel(acc, a0))
        assert typical / 10 < acc_med < typical * 10
        assert np.median(np.abs(pot - p0) / np.abs(p0)) < typical * 10
        assert np.median(_rel(jerk, j0)) > acc_med


def _forces_with_state(gpu, prec, m, r, v, eps, idx, a0, j0, **kw):
    n = len(m)
    with gpu.Context(prec, **kw) as ctx:
        ctx.set_state(m, r, v, a0, j0, np.zeros(n), np.full(n, 1.0 / 16), eps, 0.02)
        ctx.predict(0.0)
        return ctx.force(idx)


@pytest.mark.parametrize("n,n_act", [(4096, 4096), (8192, 700), (20000, 20000)])
def test_hybrid_spj_jerk_within_plain_sum_bound(gpu, orc, n, n_act):
    """HYBRID_SPJ: the far pairs' jerk in one plain FP32 sum per warp; its
    jerk within (16 + N) u sum |j_ij| of the oracle, and acceleration and
    potential bit-identical to HYBRID under the same launch shape."""
    m, r, v = ics.plummer(n, 40 + n)
    eps = 4.0 / n
    idx = ics.permutation(n, 14)[:n_act].astype(np.int32)
    a_all, j_all, _ = orc.force(m, r, v, eps, nthreads=NTHREADS)
    shape = dict(i_per_thread=2, j_split=1, ctas_per_sm=3)
    a1, j1, p1 = _forces_with_state(gpu, "hybrid", m, r, v, eps, idx, a_all, j_all, **shape)
    a2, j2, p2 = _forces_with_state(gpu, "hybrid_spj", m, r, v, eps, idx, a_all, j_all, **shape)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    _, sj, _ = _magnitude_sums(m, r, v, eps, idx)
    assert np.all(np.linalg.norm(j2 - j_all[idx], axis=1) <= (16 + n) * U32 * sj)
    if n_act == n:
        assert not np.array_equal(j1, j2)
