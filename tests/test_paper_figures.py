"""Figures the paper states (tests/golden/paper_figures.json, each cited)
against this project: the conventions the benchmark uses, and the accuracy
of the paper's own precision scheme as the CPU loop of baseline/ restates
it (Sec. 4, Fig. err_snp)."""
import json
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "paper_figures.json")) as fh:
    GOLD = json.load(fh)
NTHREADS = os.cpu_count() or 1


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def test_benchmark_uses_the_paper_conventions():
    import bench
    assert bench.FLOPS_PER_INTERACTION == GOLD["flops_per_interaction"]["value"]
    assert bench.CROSSING_TIME == pytest.approx(GOLD["crossing_time_nbody_units"]["value"],
                                                rel=1e-15)
    assert bench.ENERGY_STUDY_T_END == GOLD["energy_study_end_time"]["value"]


def test_paper_scheme_accuracy_matches_fig_err_snp(orc):
    """Plummer models, eps = 4/N, 256 sampled i against all j: accelerations
    within a factor of 10 of the stated 1e-8 at the median, potentials no
    worse, jerks less accurate than accelerations, and (single-precision jerk
    sums) the jerk error growing from N = 1K to 16K."""
    from baseline import paper_cpu
    paper_cpu.build()
    typical = GOLD["acc_pot_relative_error_typical"]["value"]
    jerk_med = {}
    for n in (1024, 16384):
        m, r, v = ics.plummer(n, 11)
        eps = 4.0 / n
        idx = ics.permutation(n, 2)[:256].astype(np.int32)
        a, j, p = paper_cpu.force(m, r, v, eps, idx, nthreads=NTHREADS)
        a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
        acc_med = np.median(_rel(a, a0))
        pot_med = np.median(np.abs(p - p0) / np.abs(p0))
        jerk_med[n] = np.median(_rel(j, j0))
        assert typical / 10 < acc_med < typical * 10
        assert pot_med < typical * 10
        assert GOLD["jerk_less_accurate_than_acc"]["value"] and jerk_med[n] > acc_med
    assert GOLD["jerk_error_grows_with_n_under_sp_sums"]["value"]
    assert jerk_med[16384] > jerk_med[1024]
