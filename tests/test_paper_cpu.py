"""The paper-style CPU force loop (baseline/paper_cpu_force.c: Sec. 3.2-3.3
mixed precision, 2 i x 4 j per vector) against the FP64 oracle.

Tolerances: each pair term is formed in single precision from a relative
position rounded once from double (u = 2^-24 per operation, the Newton-
refined reciprocal square root within 3 u), so acceleration and potential,
summed in double, err by at most 16 u sum_j |term_ij|; the jerk, summed in
single precision over all N j, by at most (16 + N) u sum_j |jerk_ij|.
"""
import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def pcf():
    from baseline import paper_cpu
    paper_cpu.build()
    return paper_cpu


def _sums(m, r, v, eps, idx):
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


@pytest.mark.parametrize("n,n_act", [(2, 2), (7, 5), (64, 64), (1001, 333)])
def test_paper_cpu_within_mixed_bounds(pcf, orc, n, n_act):
    m, r, v = ics.plummer(n, 40 + n) if n > 2 else (
        np.array([0.6, 0.4]), np.array([[0.1, 0.0, 0.0], [-0.2, 0.3, 0.1]]),
        np.array([[0.0, 0.2, 0.0], [0.1, -0.1, 0.3]]))
    eps = 4.0 / n if n > 2 else 0.01
    idx = ics.permutation(n, 3)[:n_act].astype(np.int32)
    acc, jerk, pot = pcf.force(m, r, v, eps, idx, nthreads=2)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=2)
    sa, sj, sp = _sums(m, r, v, eps, idx)
    assert np.all(np.linalg.norm(acc - a0, axis=1) <= 16 * U32 * sa)
    assert np.all(np.linalg.norm(jerk - j0, axis=1) <= (16 + n) * U32 * sj)
    assert np.all(np.abs(pot - p0) <= 16 * U32 * sp)


def test_paper_cpu_two_body_closed_form(pcf):
    """a = G m_j r / (r^2 + eps^2)^(3/2), phi = -G m_j / sqrt(r^2 + eps^2)."""
    m = np.array([2.0, 0.5])
    r = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
    v = np.zeros((2, 3))
    eps, G = 0.05, 1.5
    acc, jerk, pot = pcf.force(m, r, v, eps, np.array([0, 1], np.int32), G=G, nthreads=1)
    d = r[1] - r[0]
    s2 = d @ d + eps * eps
    np.testing.assert_allclose(acc[0], G * m[1] * d / s2 ** 1.5, rtol=1e-6)
    np.testing.assert_allclose(acc[1], -G * m[0] * d / s2 ** 1.5, rtol=1e-6)
    np.testing.assert_allclose(pot, [-G * m[1] / s2 ** 0.5, -G * m[0] / s2 ** 0.5], rtol=1e-6)
    assert np.all(jerk == 0)


def test_paper_cpu_thread_count_does_not_change_results(pcf):
    n = 500
    m, r, v = ics.plummer(n, 9)
    lay = pcf.Layout(m, r, v)
    one = lay.force(4.0 / n, nthreads=1)
    many = lay.force(4.0 / n, nthreads=4)
    for x, y in zip(one, many):
        assert np.array_equal(x, y)


def test_paper_cpu_rejects_bad_index(pcf):
    m, r, v = ics.plummer(10, 1)
    with pytest.raises(ValueError):
        pcf.force(m, r, v, 0.1, np.array([3, 10], np.int32))
