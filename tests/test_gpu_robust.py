"""Failure handling and checkpoint/resume, with no GPU fault.

* A force kernel that gives up waiting for a staged j tile reports
  NB_ETIMEOUT, drains its own copies first, and leaves the context usable.
  The wait runs out because the tile is never staged (nb_selftest_timeout),
  not because of a fault.
* nb_get_state / nb_set_state is a checkpoint: a run resumed from it is bit
  for bit the run that never stopped.
"""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1


@pytest.mark.parametrize("prec", ["mixed", "ds", "fp64"])
def test_wait_timeout_reports_and_context_stays_usable(gpu, orc, prec):
    """A tile wait that nothing completes runs out; the host sees NB_ETIMEOUT
    and the same context then gives the oracle's forces."""
    n = 2000
    m, r, v = ics.plummer(n, 41)
    eps = 4.0 / n
    idx = np.arange(0, n, 7, dtype=np.int32)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    with gpu.Context(prec) as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        assert gpu.nb_selftest_timeout(ctx.handle) == gpu.NB_ETIMEOUT
        ctx.predict(0.0)
        acc, jerk, pot = ctx.force(idx)
        ctx.synchronize()
    rel = np.linalg.norm(acc - a0, axis=1) / np.linalg.norm(a0, axis=1)
    assert rel.max() < (1e-4 if prec == "mixed" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "ds"])
def test_checkpoint_resume_is_bitwise(gpu, prec):
    n = 1024
    m, r, v = ics.plummer(n, 1)
    eps, eta = 1.0 / 64, 0.02
    t1, t2 = 1.0 / 8, 1.0 / 4
    with gpu.Context(prec) as a:
        a.set_particles(m, r, v, eps, eta)
        a.step_until(t1)
        ck = a.get_state()
        a.step_until(t2)
        final_a = a.get_state()
    with gpu.Context(prec) as b:
        b.set_state(m, ck["r"], ck["v"], ck["a"], ck["j"], ck["t"], ck["dt"], eps, eta)
        b.step_until(t2)
        final_b = b.get_state()
    for k in final_a:
        assert np.array_equal(final_a[k], final_b[k]), k
    assert np.all(final_a["t"] == t2)


@pytest.mark.parametrize("prec", ["ds", "hybrid"])
def test_snapshot_restore_replays_bitwise(gpu, prec):
    """nb_snapshot / nb_restore: rolling back on the device and integrating
    again reproduces the first run bit for bit."""
    import torch
    n = 1024
    m, r, v = ics.plummer(n, 4)
    with gpu.Context(prec) as ctx:
        ctx.set_particles(m, r, v, 1.0 / 64, 0.02)
        nbytes = ctx.snapshot_bytes()
        # the state (17 words per particle and the bounds) and its spatial order
        assert nbytes == (18 * n + 1) * 8
        buf = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
        ctx.snapshot(buf)
        first = ctx.step_until(1.0 / 16)
        s1 = ctx.get_state()
        ctx.restore(buf)
        again = ctx.step_until(1.0 / 16)
        s2 = ctx.get_state()
    assert first == again
    for k in s1:
        assert np.array_equal(s1[k], s2[k]), k
