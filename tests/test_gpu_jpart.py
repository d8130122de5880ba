"""The j-partitioned force on one GPU: the parts of the j sum (nb_set_j_part)
add up to the whole force, and two contexts run as the two ranks of a
j-partitioned integration (their parts summed on the host, as the
all-reduce would) stay identical to each other and follow the oracle."""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics, jpart

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1
BOUND = {"fp64": 1e-10, "ds": 1e-9, "hybrid": 1e-6}


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("prec", ["fp64", "ds", "hybrid"])
@pytest.mark.parametrize("n,parts", [(3001, 2), (3001, 3), (700, 11)])
def test_parts_add_up_to_the_whole(gpu, orc, prec, n, parts):
    eps = 4.0 / n
    m, r, v = ics.plummer(n, 90 + parts)
    a0, j0, p0 = orc.force(m, r, v, eps, nthreads=NTHREADS)
    idx = ics.permutation(n, 4)[:n // 2].astype(np.int32)
    tot = [np.zeros((len(idx), 3)), np.zeros((len(idx), 3)), np.zeros(len(idx))]
    for part in range(parts):
        with gpu.Context(prec) as ctx:
            # the hybrid near-pair test reads the state's a, j
            ctx.set_state(m, r, v, a0, j0, np.zeros(n), np.full(n, 1.0 / 16), eps, 0.02)
            ctx.set_j_part(part, parts)
            ctx.predict(0.0)
            for t, x in zip(tot, ctx.force(idx)):
                t += x
    assert _rel(tot[0], a0[idx]).max() < BOUND[prec]
    assert _rel(tot[1], j0[idx]).max() < BOUND[prec]
    assert (np.abs(tot[2] - p0[idx]) / np.abs(p0[idx])).max() < BOUND[prec]


def test_two_rank_integration_emulated_on_one_gpu(gpu, orc):
    """Ranks 0 and 1 of a j-partitioned DS integration, each a context with
    the whole state, stepped in lockstep: select, predict, own part of the
    force, the two parts summed, correct.  Both replicas end identical, with
    the oracle's energy drift (within 2x) and block steps (within 2 %)."""
    n, eps, eta, t_end = 1024, 1.0 / 64, 0.02, 1.0 / 8
    m, r, v = ics.plummer(n, 1)
    ranks = [gpu.Context("ds") for _ in range(2)]
    try:
        for ctx in ranks:
            ctx.set_particles(m, r, v, eps, eta)
        e_start = ranks[0].energy(fp64_potential=True)
        steps = [jpart.BlockStep(ctx, k, 2, device_arrays=False) for k, ctx in enumerate(ranks)]
        blocks = 0
        while True:
            parts = [s.begin(t_end) for s in steps]
            if parts[0] is None:
                assert parts[1] is None
                break
            total = parts[0] + parts[1]
            for s in steps:
                s.finish(total)
            blocks += 1
        st = [ctx.get_state() for ctx in ranks]
        for key in st[0]:
            assert np.array_equal(st[0][key], st[1][key]), key
        assert np.all(st[0]["t"] == t_end)
        e_end = ranks[0].energy(fp64_potential=True)
    finally:
        for ctx in ranks:
            ctx.close()
    s = orc.State(m, r, v, eps, eta, nthreads=NTHREADS)
    e0 = s.energy()
    assert s.run(t_end) == orc.OK
    de_orc = abs(s.energy() - e0) / abs(e0)
    de = abs(sum(e_end) - sum(e_start)) / abs(sum(e_start))
    assert de <= 2 * de_orc + 1e-13
    assert blocks == pytest.approx(s.n_steps, rel=0.02)
    assert np.max(np.abs(st[0]["r"] - s.r)) < 1e-7


def test_j_part_rejects_bad_arguments(gpu):
    m, r, v = ics.plummer(200, 3)
    with gpu.Context("ds") as ctx:
        ctx.set_particles(m, r, v, 0.02, 0.02)
        for part, parts in ((2, 2), (-1, 2), (0, 0), (0, 5)):  # 200 particles: 4 tiles
            with pytest.raises(gpu.NbError) as e:
                ctx.set_j_part(part, parts)
            assert e.value.status == gpu.NB_EINVAL
        ctx.set_j_part(1, 4)
        off = np.array([0, 100, 200])
        ctx.set_ensemble(off, m, r, v, np.full(2, 0.02), 0.02)
        with pytest.raises(gpu.NbError) as e:
            ctx.set_j_part(0, 2)
        assert e.value.status == gpu.NB_EINVAL
