"""j-partitioned force across processes, one GPU each, for one system.

The paper's parallel runs (Sec. 4-5) split the j sum of Eqs. acc, jrk and
pot over processes.  Here every rank holds the whole Hermite state of the
system (replicated) and evaluates the force on the active block from its own
part of the j tiles (``nb_set_j_part``); the parts are summed by one
all-reduce of the block's 7 n_act values (acc, jerk, pot) per block step, and
every rank applies the same corrector to the summed forces, so the replicas
stay identical.  Selecting the block, predicting and correcting are O(N) and
run on every rank; only the O(n_act N) force is divided.

A block step is two phases so that the reduction can sit between them:
``begin`` (step 1 select, steps 2-3 predict, step 4 on this rank's j part)
and ``finish`` (steps 5-8 with the summed forces).  ``JPartitionedStepper``
runs them around ``torch.distributed.all_reduce``.
"""
from __future__ import annotations

import numpy as np

TILE = 64  # j particles per tile of the library's j layout


def j_tile_range(part: int, parts: int, n_tiles: int):
    """Tiles [lo, hi) of part `part` of `parts` (the library's formula)."""
    if not (parts >= 1 and 0 <= part < parts):
        raise ValueError(f"part {part} of {parts}")
    return n_tiles * part // parts, n_tiles * (part + 1) // parts


def j_members(order: np.ndarray, part: int, parts: int) -> np.ndarray:
    """The particles whose j slot lies in part `part` of `parts`: slots
    [64 lo, 64 hi) of the stored order `order` (n particles; the ghosts that
    pad the last tile hold no particle)."""
    n = len(order)
    lo, hi = j_tile_range(part, parts, -(-n // TILE))
    return np.asarray(order[TILE * lo:min(n, TILE * hi)])


class BlockStep:
    """The two phases of one j-partitioned block step on one context."""

    def __init__(self, ctx, part: int, parts: int, device_arrays: bool):
        self.ctx = ctx
        self.device = device_arrays
        ctx.set_j_part(part, parts)
        self.t_next = None
        self.idx = None

    def begin(self, t_end):
        """Select the block due next (the same on every rank), predict, and
        evaluate this part's sums.  Returns one array of 7 n_act values
        (acc, jerk, pot) to be summed over the parts, or None when no block
        is due within t_end."""
        t_next, idx = self.ctx.select(t_end)
        if len(idx) == 0:
            return None
        self.ctx.predict(t_next)
        self.t_next = t_next
        k = len(idx)
        if self.device:
            import torch
            dev = torch.device("cuda", self.ctx.cfg.device)
            self.idx = torch.from_numpy(idx).to(dev)
            buf = torch.empty(7 * k, dtype=torch.float64, device=dev)
            acc, jerk, pot = buf[:3 * k].view(k, 3), buf[3 * k:6 * k].view(k, 3), buf[6 * k:]
            self.ctx.force(self.idx, acc, jerk, pot)
            self.ctx.synchronize()  # the context's stream is not torch's
            return buf
        self.idx = idx
        acc, jerk, pot = self.ctx.force(idx)
        return np.concatenate([acc.ravel(), jerk.ravel(), pot])

    def finish(self, summed):
        """Steps 5-8 of the block with the forces summed over every part."""
        k = len(self.idx)
        acc, jerk = summed[:3 * k].reshape(k, 3), summed[3 * k:6 * k].reshape(k, 3)
        self.ctx.correct(self.t_next, self.idx, acc, jerk)
        return k


class JPartitionedStepper:
    """Integrate one system over the ranks of a torch.distributed group:
    rank r sums the j tiles of part r of world_size.  With the NCCL backend
    the block's forces stay on the GPU; with gloo they travel as host
    arrays."""

    def __init__(self, ctx, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        self.device = dist.get_backend(group) == "nccl"
        self.step = BlockStep(ctx, rank, world, self.device)
        self.n = ctx.n

    def block_step(self, t_end) -> int:
        """One block step; returns its n_act (0 once no block is due)."""
        import torch
        part = self.step.begin(t_end)
        if part is None:
            return 0
        t = part if self.device else torch.from_numpy(part)
        self.dist.all_reduce(t, group=self.group)
        if self.device:
            torch.cuda.current_stream().synchronize()  # before the context's stream reads it
        return self.step.finish(t if self.device else t.numpy())

    def step_until(self, t_end):
        """Block steps until none is due within t_end: (steps, interactions)."""
        steps = inter = 0
        while True:
            k = self.block_step(t_end)
            if k == 0:
                return steps, inter
            steps += 1
            inter += k * self.n
