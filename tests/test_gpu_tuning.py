"""Launch shapes set by hand (nb_set_tuning) and the block-size windows of
one system.

A force call whose block size the host knows goes to one launch: the tiny
shape below tiny_split, the small one below nact_split, the large one
above.  A block step, whose size is on the device, launches the small and
the large shape as parallel branches, of which the one whose window holds
n_act works, and never the tiny shape.  These cases check each window
against the FP64 oracle, which shape each path takes (bit for bit against a
context whose small shape is the tiny one), and the argument checks."""
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1
BOUND = {"ds": 1e-9, "hybrid": 1e-6}


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _shapes(tiny_split=64, tiny_j_split=8, small_j_split=4, large_j_split=2, cps=2):
    return dict(small_i_per_thread=1, small_j_split=small_j_split, small_ctas_per_sm=cps,
                large_i_per_thread=1, large_j_split=large_j_split, large_ctas_per_sm=cps,
                nact_split=1024, tiny_split=tiny_split, tiny_i_per_thread=1,
                tiny_j_split=tiny_j_split, tiny_ctas_per_sm=cps)


@pytest.fixture(scope="module")
def plummer8k():
    n = 8192
    m, r, v = ics.plummer(n, 41)
    return m, r, v, 4.0 / n


@pytest.mark.parametrize("prec", ["hybrid", "ds"])
def test_three_windows_against_oracle(gpu, orc, plummer8k, prec):
    m, r, v, eps = plummer8k
    n = len(m)
    perm = ics.permutation(n, 9).astype(np.int32)
    with gpu.Context(prec) as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        ctx.set_tuning(**_shapes())
        ctx.predict(0.0)
        # both edges of each window: tiny [0, 64), small [64, 1024), large
        for k in (1, 63, 64, 500, 1023, 1024, 3000):
            idx = np.sort(perm[:k])
            a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
            acc, jerk, pot = ctx.force(idx)
            assert _rel(acc, a0).max() < BOUND[prec], k
            assert _rel(jerk, j0).max() < BOUND[prec], k
            assert (np.abs(pot - p0) / np.abs(p0)).max() < BOUND[prec], k


def _integrate(gpu, m, r, v, eps, shapes, t_end=1.0 / 64):
    with gpu.Context("hybrid") as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        ctx.set_tuning(**shapes)
        steps, inter = ctx.step_until(t_end)
        return steps, inter, ctx.get_state()


def test_block_steps_never_take_the_tiny_shape(gpu, plummer8k):
    """Device-sized block steps with a tiny shape of its own (j split 8
    against the small blocks' 4) give every bit of the run without one."""
    m, r, v, eps = plummer8k
    with_tiny = _integrate(gpu, m, r, v, eps, _shapes(tiny_split=160, tiny_j_split=8))
    without = _integrate(gpu, m, r, v, eps, _shapes(tiny_split=0))
    assert with_tiny[0] == without[0] and with_tiny[1] == without[1] and without[0] > 0
    for key in ("r", "v", "a", "j", "t", "dt"):
        assert np.array_equal(with_tiny[2][key], without[2][key]), key


@pytest.mark.parametrize("prec", ["hybrid", "mixed"])
def test_host_sized_force_takes_the_tiny_shape(gpu, plummer8k, prec):
    """Below tiny_split a host-sized force call runs the tiny shape: its
    results match, bit for bit, a context whose small shape is that shape."""
    m, r, v, eps = plummer8k
    idx = np.sort(ics.permutation(len(m), 3)[:40]).astype(np.int32)
    out = []
    for shapes in (_shapes(tiny_split=64, tiny_j_split=8, small_j_split=2),
                   _shapes(tiny_split=0, small_j_split=8)):
        with gpu.Context(prec) as ctx:
            ctx.set_particles(m, r, v, eps, 0.02)
            ctx.set_tuning(**shapes)
            ctx.predict(0.0)
            out.append(ctx.force(idx))
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_set_tuning_rejects_bad_shapes(gpu, plummer8k):
    m, r, v, eps = plummer8k
    bad = [dict(tiny_split=1024), dict(tiny_split=-1), dict(tiny_j_split=3),
           dict(cps=0), dict(cps=99)]
    with gpu.Context("hybrid") as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        for kw in bad:
            with pytest.raises(gpu.NbError) as e:
                ctx.set_tuning(**_shapes(**kw))
            assert e.value.status == gpu.NB_EINVAL, kw
        with pytest.raises(gpu.NbError) as e:  # two i per thread take no j split
            ctx.set_tuning(**dict(_shapes(), small_i_per_thread=2))
        assert e.value.status == gpu.NB_EINVAL
        for chunks in (-1, 5):  # stream-K chunks per warp: 0 (default) to 4
            with pytest.raises(gpu.NbError) as e:
                ctx.set_tuning(**dict(_shapes(), ens_chunks=chunks))
            assert e.value.status == gpu.NB_EINVAL
        ctx.set_tuning(**_shapes(tiny_split=0, tiny_j_split=0))  # tiny unused: unchecked
        ctx.predict(0.0)
        ctx.force(np.arange(10, dtype=np.int32))  # the errors were not sticky
    offsets = np.array([0, 4096, 8192], dtype=np.int64)
    with gpu.Context("hybrid") as ctx:
        ctx.set_ensemble(offsets, m, r, v, np.array([eps, eps]), 0.02)
        with pytest.raises(gpu.NbError) as e:
            ctx.set_tuning(**_shapes())
        assert e.value.status == gpu.NB_EINVAL
        with pytest.raises(gpu.NbError) as e:
            ctx.set_tuning(**_shapes(tiny_split=0))  # small and large j splits differ
        assert e.value.status == gpu.NB_EINVAL
        ctx.set_tuning(**_shapes(tiny_split=0, small_j_split=2))
        steps, _ = ctx.step_until(1.0 / 256)
        assert steps > 0


def test_autotuned_shapes_round_trip(gpu, plummer8k):
    """The autotuner's choice, set again by hand, gives the same forces."""
    m, r, v, eps = plummer8k
    idx = np.arange(0, 8192, 61, dtype=np.int32)
    with gpu.Context("hybrid") as ctx:
        ctx.set_particles(m, r, v, eps, 0.02)
        tun = ctx.autotune()
        assert tun["tiny_split"] in (0, 64, 160)
        if tun["tiny_split"]:
            assert tun["tiny_i_per_thread"] in (1, 2) and tun["tiny_us"] > 0
            assert tun["tiny_j_split"] in (1, 2, 4, 8) and tun["tiny_ctas_per_sm"] >= 1
        ctx.set_particles(m, r, v, eps, 0.02)
        ctx.predict(0.0)
        ref = [ctx.force(idx[:k]) for k in (5, 100, len(idx))]
        ctx.set_tuning(**tun)
        ctx.set_particles(m, r, v, eps, 0.02)  # the same noise estimates again
        ctx.predict(0.0)
        out = [ctx.force(idx[:k]) for k in (5, 100, len(idx))]
    for a, b in zip(ref, out):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
