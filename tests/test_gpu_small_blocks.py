"""Small blocks of large systems against the oracle.

A block with at most a quarter as many i-groups as CTAs is summed CTA by
CTA: each CTA's four warps in shared memory, then the CTAs' entries in a
tree whose chunks the last CTA of each adds.  At N = 65536 a block of a few
particles spans up to 256 CTAs, so the tree has two levels; these cases
(one i per lane with j splits of 1 and 8, device and host index lists)
check every result against the FP64 oracle, and the j windows of a
j-partitioned force on such blocks."""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1
BOUND = {"fp64": 1e-10, "ds": 1e-9, "hybrid": 1e-6, "mixed": 2e-5}


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.fixture(scope="module")
def n64k():
    wl = ics.MIXED_N64K
    m, r, v = wl.particles()
    return m, r, v, wl.eps


@pytest.mark.parametrize("prec", ["hybrid", "ds"])
@pytest.mark.parametrize("j_split", [1, 8])
@pytest.mark.parametrize("n_act", [1, 8, 40, 200])
def test_small_block_n65536_against_oracle(gpu, orc, n64k, prec, j_split, n_act):
    m, r, v, eps = n64k
    n = len(m)
    idx = ics.permutation(n, 31 + n_act)[:n_act].astype(np.int32)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    torch = pytest.importorskip("torch")
    with gpu.Context(prec, j_split=j_split) as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        ctx.predict(0.0)
        snap = torch.empty(ctx.snapshot_bytes() // 8 + 1, dtype=torch.float64, device="cuda")
        ctx.snapshot(snap)
        acc, jerk, pot = ctx.force(idx)
        # again from the same state (the hybrid noise estimates included):
        # the reduction's counters were left at zero, the sums in fixed order
        ctx.restore(snap)
        ctx.predict(0.0)
        acc2, jerk2, pot2 = ctx.force(idx)
    assert _rel(acc, a0).max() < BOUND[prec] and _rel(jerk, j0).max() < BOUND[prec]
    assert (np.abs(pot - p0) / np.abs(p0)).max() < BOUND[prec]
    assert np.array_equal(acc, acc2) and np.array_equal(jerk, jerk2) and np.array_equal(pot, pot2)


def test_small_block_device_list_n65536(gpu, orc, n64k):
    """A device index list in the caller's numbering (mapped to the stored
    order by the kernel) gives the host list's results, row for row."""
    torch = pytest.importorskip("torch")
    m, r, v, eps = n64k
    n = len(m)
    idx = ics.permutation(n, 77)[:24].astype(np.int32)
    with gpu.Context("hybrid") as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        ctx.predict(0.0)
        ref = ctx.force(idx)
        di = torch.from_numpy(idx).cuda()
        out = [torch.empty((24, 3), dtype=torch.float64, device="cuda"),
               torch.empty((24, 3), dtype=torch.float64, device="cuda"),
               torch.empty(24, dtype=torch.float64, device="cuda")]
        ctx.force(di, *out)
        ctx.synchronize()
    for x, y in zip(ref, out):
        assert np.array_equal(x, y.cpu().numpy())


@pytest.mark.parametrize("parts", [2, 5])
def test_small_block_j_parts_add_up(gpu, orc, n64k, parts):
    m, r, v, eps = n64k
    n = len(m)
    idx = ics.permutation(n, 5)[:16].astype(np.int32)
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    tot = [np.zeros((16, 3)), np.zeros((16, 3)), np.zeros(16)]
    for part in range(parts):
        with gpu.Context("ds") as ctx:
            ctx.set_particles(m, r, v, eps, 0.02)
            ctx.set_j_part(part, parts)
            ctx.predict(0.0)
            for t, x in zip(tot, ctx.force(idx)):
                t += x
    assert _rel(tot[0], a0).max() < 1e-9 and _rel(tot[1], j0).max() < 1e-9
    assert (np.abs(tot[2] - p0) / np.abs(p0)).max() < 1e-9
