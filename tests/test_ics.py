"""Seeded synthetic inputs: Plummer model (Sec. 4-5 workloads), Salpeter masses."""
import math

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics


def test_counter_rng_is_deterministic_and_uniform():
    a = ics.uniform(5, np.arange(100000, dtype=np.uint64))
    b = ics.uniform(5, np.arange(100000, dtype=np.uint64))
    assert np.array_equal(a, b)
    assert 0.0 < a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.005
    assert not np.array_equal(a, ics.uniform(6, np.arange(100000, dtype=np.uint64)))


def test_splitmix64_reference_value():
    # SplitMix64 with state 0: the first output of the published generator.
    z = ics._mix64(np.uint64(0) + ics.GAMMA)
    assert int(z) == 0xE220A8397B1DCDAF


def test_plummer_centre_of_mass_and_scaling():
    m, r, v = ics.plummer(4096, 3)
    assert m.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose((m[:, None] * r).sum(0), 0.0, atol=1e-14)
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0.0, atol=1e-14)


def test_plummer_cumulative_mass_profile_ks():
    stats = pytest.importorskip("scipy.stats")
    n = 8192
    m, r, v = ics.plummer(n, 4)
    a = 3 * math.pi / 16  # Plummer scale length in standard N-body units
    rad = np.linalg.norm(r - np.average(r, axis=0, weights=m), axis=1)
    rcut = 10 * a
    mcut = rcut ** 3 / (rcut ** 2 + a ** 2) ** 1.5

    def cdf(x):
        x = np.minimum(x, rcut)
        return x ** 3 / (x ** 2 + a ** 2) ** 1.5 / mcut

    # the centre-of-mass shift is O(1/sqrt(N)); compare the raw radii
    _, p = stats.kstest(rad, cdf)
    assert p > 1e-3


def test_plummer_virial_and_energy(orc):
    # The r <= 10 a truncation keeps the outer 1.5 % of the mass inside the
    # cut while speeds follow the untruncated model, so E sits near -0.26
    # rather than -1/4; N = 2048 adds a few per cent of sampling noise.
    m, r, v = ics.plummer(2048, 5)
    K, W = orc.energy(m, r, v, eps=0.0, nthreads=4)
    assert 2 * K / abs(W) == pytest.approx(1.0, abs=0.06)
    assert -0.285 < K + W < -0.24


def test_salpeter_moment_ratio_matches_closed_form():
    n = 200000
    m = ics.salpeter_masses(n, 9)
    assert m.sum() == pytest.approx(1.0, rel=1e-12)
    s, lo, hi = 2.35, 0.1, 10.0

    def mom(k):
        p = k + 1 - s
        return (hi ** p - lo ** p) / p

    ratio = mom(2) * mom(0) / mom(1) ** 2  # E[m^2] / E[m]^2, scale free
    sample = np.mean(m ** 2) / np.mean(m) ** 2
    assert sample == pytest.approx(ratio, rel=0.05)
    assert m.max() / m.min() <= 100.0 + 1e-9


def test_permutation_and_ensemble_sizes():
    p = ics.permutation(1000, 2)
    assert sorted(p) == list(range(1000))
    sizes = ics.ensemble_sizes(256, 4)
    assert sizes.min() >= 256 and sizes.max() <= 8192
    lg = np.log(sizes)
    assert abs(lg.mean() - 0.5 * (math.log(256) + math.log(8192))) < 0.3
