"""The sixth-order Hermite variant (NB_FP64_HERMITE6; adjacent to the paper,
which integrates with the fourth-order scheme) against its FP64 oracle: the
snap of the force kernel, and block-timestep integrations."""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("n,eps", [(64, 1 / 64), (1000, 4 / 1000), (4097, 4 / 4097)])
def test_load_snap_equals_oracle(gpu, orc, n, eps):
    """After nb_set_particles every particle carries a, j from the load and
    the snap of a second pass with those accelerations (reading H3): the
    FP64 kernel's acc, jerk, snap and pot within 1e-10 of the oracle's."""
    m, r, v = ics.plummer(n, 70 + n)
    with gpu.Context("fp64_hermite6") as ctx:
        ctx.set_particles(m, r, v, eps, 0.1)
        st = ctx.get_state()
        snap, crackle = ctx.get_snap()
        ctx.predict(0.0)
        idx = ics.permutation(n, 2)[:min(n, 500)].astype(np.int32)
        acc, jerk, pot = ctx.force(idx)
    a0, j0, p0 = orc.force(m, r, v, eps, nthreads=NTHREADS)
    a1, j1, s1, p1 = orc.force_snap(m, r, v, a0, eps, nthreads=NTHREADS)
    assert _rel(st["a"], a0).max() < 1e-10 and _rel(st["j"], j0).max() < 1e-10
    assert _rel(snap, s1).max() < 1e-10
    assert np.all(crackle == 0.0)
    assert _rel(acc, a1[idx]).max() < 1e-10 and _rel(jerk, j1[idx]).max() < 1e-10
    assert (np.abs(pot - p1[idx]) / np.abs(p1[idx])).max() < 1e-10


@pytest.mark.parametrize("n,eps,eta,t_end", [(256, 1 / 64, 0.1, 0.25), (1024, 1 / 64, 0.1, 0.125)])
def test_integration_matches_oracle(gpu, orc, n, eps, eta, t_end):
    """Plummer models integrated with the sixth-order scheme on the GPU and by
    the oracle: the same block steps (within 1 %) and interactions, energy
    drift within 2x the oracle's, final positions within 1e-9."""
    m, r, v = ics.plummer(n, 1)
    s = orc.State6(m, r, v, eps, eta, nthreads=NTHREADS)
    e0 = s.energy()
    assert s.run(t_end) == orc.OK
    de_orc = abs(s.energy() - e0) / abs(e0)
    with gpu.Context("fp64_hermite6") as ctx:
        ctx.set_particles(m, r, v, eps, eta)
        steps, inter = ctx.step_until(t_end)
        k1, w1 = ctx.energy(fp64_potential=True)
        out = ctx.get_state()
    de = abs(k1 + w1 - e0) / abs(e0)
    assert np.all(out["t"] == t_end)
    assert steps == pytest.approx(s.n_steps, rel=0.01)
    assert inter == pytest.approx(s.n_inter, rel=0.01)
    assert de <= 2 * de_orc + 1e-13, (de, de_orc)
    assert np.max(np.abs(out["r"] - s.r)) < 1e-9


def test_sixth_order_reaches_fourth_order_energy_in_fewer_steps(gpu):
    """The N = 1024 workload to t = 0.5: the sixth-order scheme at eta = 0.1
    conserves energy at least as well as the fourth-order scheme at
    eta = 0.02 with fewer block steps."""
    n, eps = 1024, 1.0 / 64
    m, r, v = ics.plummer(n, 1)
    res = {}
    for prec, eta in (("fp64", 0.02), ("fp64_hermite6", 0.1)):
        with gpu.Context(prec) as ctx:
            ctx.set_particles(m, r, v, eps, eta)
            k0, w0 = ctx.energy(fp64_potential=True)
            steps, _ = ctx.step_until(0.5)
            k1, w1 = ctx.energy(fp64_potential=True)
        res[prec] = (steps, abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0))
    assert res["fp64_hermite6"][0] < res["fp64"][0]
    assert res["fp64_hermite6"][1] < 2 * res["fp64"][1], res


def test_sixth_order_restrictions(gpu):
    m, r, v = ics.plummer(200, 3)
    with gpu.Context("fp64_hermite6") as ctx:
        ctx.set_particles(m, r, v, 0.02, 0.1)
        with pytest.raises(gpu.NbError) as e:
            ctx.set_ensemble(np.array([0, 100, 200]), m, r, v, np.full(2, 0.02), 0.1)
        assert e.value.status == gpu.NB_EINVAL
        st = ctx.get_state() if ctx.n else None
    with gpu.Context("fp64_hermite6") as ctx:
        t = np.zeros(200)
        t[5] = 1.0 / 16
        with pytest.raises(gpu.NbError) as e:
            ctx.set_state(m, r, v, np.zeros((200, 3)), np.zeros((200, 3)), t,
                          np.full(200, 1.0 / 16), 0.02, 0.1)
        assert e.value.status == gpu.NB_EINVAL
    assert st is not None
