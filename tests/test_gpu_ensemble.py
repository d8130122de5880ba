"""Ensembles of independent systems in one context (many clusters per launch).

Pins: every system's forces equal the oracle's on that system alone, and an
ensemble integration gives each system the trajectory it has when run alone
(same precision), up to the summation order of split i-groups.
"""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1


def _systems(sizes, seed0):
    ms, rs, vs = [], [], []
    for q, n in enumerate(sizes):
        m, r, v = ics.plummer(int(n), seed0 + q)
        ms.append(m)
        rs.append(r)
        vs.append(v)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    eps = 4.0 / np.asarray(sizes, dtype=np.float64)
    return off, np.concatenate(ms), np.concatenate(rs), np.concatenate(vs), eps


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("split", [1, 4, 8])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("ds", 1e-9), ("hybrid", 1e-6)])
def test_ensemble_force_equals_each_system_alone(gpu, orc, prec, tol, split):
    """split: lanes per i (the j split inside a warp), so groups of 32 / split
    active particles and their partial sums added by warp shuffles."""
    sizes = [100, 333, 1000, 64, 2049, 1]
    off, m, r, v, eps = _systems(sizes, 300)
    n = off[-1]
    with gpu.Context(prec, j_split=split) as ctx:
        ctx.set_ensemble(off, m, r, v, eps, 0.02)
        assert gpu.nb_num_systems(ctx.handle) == len(sizes)
        ctx.predict(0.0)
        # every particle, then a sparse ascending subset
        for idx in (np.arange(n, dtype=np.int32),
                    np.sort(ics.permutation(int(n), 5)[:777]).astype(np.int32)):
            acc, jerk, pot = ctx.force(idx)
            for q in range(len(sizes)):
                sel = (idx >= off[q]) & (idx < off[q + 1])
                if not np.any(sel):
                    continue
                lo, hi = off[q], off[q + 1]
                local = idx[sel] - lo
                a0, j0, p0 = orc.force(m[lo:hi], r[lo:hi], v[lo:hi], eps[q], idx=local,
                                       nthreads=NTHREADS)
                if hi - lo == 1:
                    assert np.all(acc[sel] == 0) and np.all(pot[sel] == 0)
                    continue
                assert _rel(acc[sel], a0).max() < tol
                assert _rel(jerk[sel], j0).max() < tol
                assert (np.abs(pot[sel] - p0) / np.abs(p0)).max() < tol


@pytest.mark.parametrize("chunks", [1, 2, 4])
@pytest.mark.parametrize("prec,tol", [("ds", 1e-9), ("hybrid", 1e-6)])
def test_ensemble_queued_chunks(gpu, orc, prec, tol, chunks):
    """Several stream-K chunks per warp, those past each warp's first handed
    out by a queue in the order warps come free.  Groups of 4 (j split 8)
    and one CTA per SM give ~23000 tiles for 608 warps, so with 4 chunks per
    warp 1824 chunks go through the queue.  Every system's forces equal the
    oracle's, in two launches in a row (a queue left non-zero by the first
    would drop chunks from the second), and the second repeats the first
    bit for bit where nothing else changed between them (DS)."""
    sizes = [100, 333, 1000, 64, 2049, 1, 700]
    off, m, r, v, eps = _systems(sizes, 500)
    n = int(off[-1])
    shape = dict(small_i_per_thread=1, small_j_split=8, small_ctas_per_sm=1,
                 large_i_per_thread=1, large_j_split=8, large_ctas_per_sm=1,
                 nact_split=1024, ens_chunks=chunks)
    idx = np.arange(n, dtype=np.int32)
    with gpu.Context(prec) as ctx:
        ctx.set_ensemble(off, m, r, v, eps, 0.02)
        ctx.set_tuning(**shape)
        ctx.predict(0.0)
        runs = [ctx.force(idx), ctx.force(idx)]
    for q in range(len(sizes)):
        lo, hi = off[q], off[q + 1]
        if hi - lo == 1:
            continue
        a0, j0, p0 = orc.force(m[lo:hi], r[lo:hi], v[lo:hi], eps[q], nthreads=NTHREADS)
        for acc, jerk, pot in runs:
            assert _rel(acc[lo:hi], a0).max() < tol, q
            assert _rel(jerk[lo:hi], j0).max() < tol, q
            assert (np.abs(pot[lo:hi] - p0) / np.abs(p0)).max() < tol, q
    if prec == "ds":
        for x, y in zip(*runs):
            assert np.array_equal(x, y)


def test_ensemble_integration_matches_each_system_alone(gpu):
    sizes = [128, 300, 512, 77]
    off, m, r, v, eps = _systems(sizes, 400)
    t_end = 1.0 / 8
    with gpu.Context("fp64") as ens:
        ens.set_ensemble(off, m, r, v, eps, 0.02)
        k0, w0 = ens.energy_systems()
        steps, inter = ens.step_until(t_end)
        k1, w1 = ens.energy_systems()
        out = ens.get_state()
    assert np.all(out["t"] == t_end)
    total_inter = 0
    max_steps = 0
    for q, nq in enumerate(sizes):
        lo, hi = off[q], off[q + 1]
        with gpu.Context("fp64") as one:
            one.set_particles(m[lo:hi], r[lo:hi], v[lo:hi], eps[q], 0.02)
            K0, W0 = one.energy()
            s_q, i_q = one.step_until(t_end)
            K1, W1 = one.energy()
            o = one.get_state()
        total_inter += i_q
        max_steps = max(max_steps, s_q)
        assert k0[q] == pytest.approx(K0, rel=1e-13) and w0[q] == pytest.approx(W0, rel=1e-12)
        # same schedule up to rounding of split sums: states agree closely
        assert np.max(np.abs(out["r"][lo:hi] - o["r"])) < 1e-9
        assert np.max(np.abs(out["v"][lo:hi] - o["v"])) < 1e-9
        assert k1[q] + w1[q] == pytest.approx(K1 + W1, rel=1e-10)
    # one ensemble block step advances every due system at once
    assert inter == total_inter
    assert max_steps <= steps <= sum(1 for _ in sizes) * max_steps


def test_ensemble_rejects_bad_input(gpu):
    off = np.array([0, 10, 10, 20], dtype=np.int64)  # empty system
    m, r, v = ics.plummer(20, 1)
    with gpu.Context("mixed") as ctx:
        with pytest.raises(gpu.NbError) as e:
            ctx.set_ensemble(off, m, r, v, np.full(3, 0.1), 0.02)
        assert e.value.status == gpu.NB_EINVAL
        ctx.set_ensemble(np.array([0, 10, 20]), m, r, v, np.full(2, 0.1), 0.02)
        with pytest.raises(gpu.NbError) as e:
            ctx.force(np.array([5, 3], dtype=np.int32))  # not ascending
        assert e.value.status == gpu.NB_EINVAL
        with pytest.raises(gpu.NbError) as e:
            ctx.correct(0.1, np.array([0], dtype=np.int32))
        assert e.value.status == gpu.NB_ESTATE


def test_hybrid_ensemble_integration_matches_oracle_per_system(gpu, orc):
    """The batched mode the benchmark times: 16 members of the ensemble
    workload integrated together in one HYBRID context (one launch per kernel
    per block step for all of them) from t = 0 to 1/16, each compared with
    the FP64 oracle's integration of that system alone (Sec. 2, steps 1-9):
      * relative energy drift within 2x the oracle's (plus 1e-13, the
        rounding of the FP64 energy sums themselves);
      * final positions within 1e-6 and velocities within 1e-5 (absolute,
        N-body units): force errors of <= 1e-6 relative move a particle by
        ~1e-6 |a| t^2, and a timestep chosen one power of two apart changes
        it by the Hermite truncation error, both far below these;
      * at least 95 % of each system's particles on the oracle's timestep,
        and the total interactions within 5 % of the oracle's sum (the
        ensemble's block steps interleave all systems, so its own step count
        is not comparable with one system's)."""
    pick, off, m, r, v, eps = ics.ensemble_subset(16, 2048)
    t_end = 1.0 / 16
    with gpu.Context("hybrid") as ens:
        ens.set_ensemble(off, m, r, v, eps, 0.02)
        steps, inter = ens.step_until(t_end)
        k1, w1 = ens.energy_systems(fp64_potential=True)
        out = ens.get_state()
    assert np.all(out["t"] == t_end)
    orc_inter = 0.0
    report = []
    for q in range(len(pick)):
        lo, hi = off[q], off[q + 1]
        s = orc.State(m[lo:hi], r[lo:hi], v[lo:hi], float(eps[q]), 0.02, nthreads=NTHREADS)
        e0 = s.energy()
        assert s.run(t_end) == orc.OK
        de_orc = abs(s.energy() - e0) / abs(e0)
        de_gpu = abs(k1[q] + w1[q] - e0) / abs(e0)
        orc_inter += s.n_inter
        dr = np.max(np.abs(out["r"][lo:hi] - s.r))
        dv = np.max(np.abs(out["v"][lo:hi] - s.v))
        same_dt = np.mean(out["dt"][lo:hi] == s.dt)
        report.append((pick[q], hi - lo, de_gpu, de_orc, dr, dv, same_dt))
        assert de_gpu <= 2.0 * de_orc + 1e-13, report[-1]
        assert dr < 1e-6 and dv < 1e-5, report[-1]
        assert same_dt >= 0.95, report[-1]
    assert inter == pytest.approx(orc_inter, rel=0.05)
