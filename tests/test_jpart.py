"""The j-partitioned force (the paper's parallel scheme splits the j sum over
processes, Sec. 4-5) on CPU: the partition of the j layout and the sum of the
parts over two gloo ranks, with the FP64 oracle as each rank's force."""
import os
import socket

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics, jpart

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 4097])
@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_parts_cover_every_particle_once(n, parts):
    order = ics.permutation(n, 3)
    tiles = -(-n // 64)
    if parts > tiles:
        with pytest.raises(ValueError):
            jpart.j_tile_range(parts, parts, tiles)
        return
    got = np.concatenate([jpart.j_members(order, p, parts) for p in range(parts)])
    assert np.array_equal(np.sort(got), np.arange(n))
    # contiguous runs of whole tiles, in the stored order
    lo, hi = jpart.j_tile_range(parts - 1, parts, tiles)
    assert hi == tiles and jpart.j_tile_range(0, parts, tiles)[0] == 0


def _partial_force(orc, m, r, v, eps, members):
    """Eqs. acc, jrk, pot on every particle i from the j in `members` only
    (j != i), by the oracle on the sub-system members + {i}."""
    n = len(m)
    inside = np.zeros(n, dtype=bool)
    inside[members] = True
    acc, jerk, pot = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    pos = {int(j): k for k, j in enumerate(members)}
    a, j, p = orc.force(m[members], r[members], v[members], eps,
                        idx=np.arange(len(members)))
    acc[members], jerk[members], pot[members] = a, j, p
    for i in np.flatnonzero(~inside):
        sub = np.append(members, i)
        a, j, p = orc.force(m[sub], r[sub], v[sub], eps, idx=[len(members)])
        acc[i], jerk[i], pot[i] = a[0], j[0], p[0]
    assert len(pos) == len(members)
    return acc, jerk, pot


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, eps = 300, 4.0 / 300
    m, r, v = ics.plummer(n, 12)
    order = ics.permutation(n, 13)  # any stored order
    a, j, p = _partial_force(oracle, m, r, v, eps, jpart.j_members(order, rank, world))
    buf = torch.from_numpy(np.concatenate([a.ravel(), j.ravel(), p]))
    dist.all_reduce(buf)
    np.save(os.path.join(out_dir, f"sum{rank}.npy"), buf.numpy())
    dist.destroy_process_group()


def test_two_rank_parts_sum_to_the_whole(tmp_path, orc):
    """Two gloo ranks, each the oracle's force from its half of the j tiles;
    their all-reduced sum is the one-rank force (to FP64 rounding)."""
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    n, eps = 300, 4.0 / 300
    m, r, v = ics.plummer(n, 12)
    a0, j0, p0 = orc.force(m, r, v, eps)
    for rank in range(2):
        got = np.load(tmp_path / f"sum{rank}.npy")
        a, j, p = got[:3 * n].reshape(n, 3), got[3 * n:6 * n].reshape(n, 3), got[6 * n:]
        assert np.max(np.linalg.norm(a - a0, axis=1) / np.linalg.norm(a0, axis=1)) < 1e-13
        assert np.max(np.linalg.norm(j - j0, axis=1) / np.linalg.norm(j0, axis=1)) < 1e-12
        assert np.max(np.abs(p - p0) / np.abs(p0)) < 1e-13


class _OracleRank:
    """A stand-in for a context, for the stepper's sequencing on CPU: the
    oracle's block-step primitives (select, predict, corrector, Eq.
    timestep, power-of-two rule) on a replicated state, and the force from
    this rank's part of the j particles only."""

    def __init__(self, orc, m, r, v, eps, eta):
        self.orc, self.m, self.eps, self.eta = orc, m, eps, eta
        s = orc.State(m, r, v, eps, eta)
        self.r, self.v, self.a, self.j, self.t, self.dt = s.r, s.v, s.a, s.j, s.t, s.dt
        self.n = len(m)
        self.order = np.arange(self.n)

    def set_j_part(self, part, parts):
        self.members = jpart.j_members(self.order, part, parts)

    def select(self, t_end):
        t_next, idx = self.orc.select(self.t, self.dt)
        return (t_next, idx.astype(np.int32)) if t_next <= t_end else (t_next, idx[:0])

    def predict(self, t):
        self.rp, self.vp = self.orc.predict(self.r, self.v, self.a, self.j, self.t, t)
        self.t_pred = t

    def force(self, idx):
        a, j, p = _partial_force(self.orc, self.m, self.rp, self.vp, self.eps, self.members)
        return a[idx], j[idx], p[idx]

    def correct(self, t, idx, acc, jerk):
        for k, i in enumerate(idx):
            h = self.dt[i]
            r1, v1, s0, c0 = self.orc.hermite_correct(self.rp[i], self.vp[i], self.a[i],
                                                      self.j[i], acc[k], jerk[k], h)
            self.r[i], self.v[i], self.a[i], self.j[i], self.t[i] = r1, v1, acc[k], jerk[k], t
            dt_a = self.orc.aarseth_dt(self.eta, self.a[i], self.j[i], s0 + c0 * h, c0)
            st, self.dt[i] = self.orc.quantize_dt(h, dt_a, t, 1.0 / 16)
            assert st == self.orc.OK


def _stepper_rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, eps, eta = 64 * 3 + 5, 1.0 / 32, 0.02
    m, r, v = ics.plummer(n, 7)
    ctx = _OracleRank(oracle, m, r, v, eps, eta)
    steps, inter = jpart.JPartitionedStepper(ctx).step_until(1.0 / 32)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), r=ctx.r, v=ctx.v, t=ctx.t, dt=ctx.dt,
             steps=steps, inter=inter)
    dist.destroy_process_group()


def test_stepper_over_two_gloo_ranks_follows_the_oracle(tmp_path, orc):
    """JPartitionedStepper on two gloo ranks (each summing half the j of a
    197-particle Plummer model, the parts all-reduced every block step):
    both replicas end identical, with the oracle's schedule and state."""
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.spawn(_stepper_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [np.load(tmp_path / f"rank{k}.npz") for k in range(2)]
    for key in ("r", "v", "t", "dt", "steps", "inter"):
        assert np.array_equal(got[0][key], got[1][key]), key
    n = 64 * 3 + 5
    m, r, v = ics.plummer(n, 7)
    ref = orc.State(m, r, v, 1.0 / 32, 0.02)
    assert ref.run(1.0 / 32) == orc.OK
    assert int(got[0]["steps"]) == ref.n_steps
    assert np.array_equal(got[0]["dt"], ref.dt) and np.array_equal(got[0]["t"], ref.t)
    assert np.max(np.abs(got[0]["r"] - ref.r)) < 1e-12
