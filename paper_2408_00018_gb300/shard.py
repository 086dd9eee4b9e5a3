"""Chains sharded over processes (one GPU each), with the exchange of the
synchronous approach (Sec. 2.2.2) between levels.

Every rank owns a contiguous block of the global chains (``shard_range``) and
runs it with a solver whose Philox chain ids are global
(``Handle.set_chain_offset``), so the numbers drawn are those of the unsharded
run.  After each level the ranks exchange their local minimum: ``minloc``
gathers every rank's (f, global chain index), keeps the lowest f (NaN never
wins, lowest index on ties) and broadcasts the owner's state; every rank then
restarts from it (``Handle.set_restart``).  The levels are then bit for bit
those of the unsharded run.

A rank that stops (exits, or never joins an exchange) surfaces on the others
as a ``ShardError`` at their next exchange: the collective fails when the
peer's connection closes, or when the process group's timeout expires.  No
device work is in flight across the exchange: every level ends with a
synchronising read of the shard's result.
"""
from __future__ import annotations

import math

import numpy as np


class ShardError(RuntimeError):
    """An exchange between shards failed (a rank stopped or timed out)."""


def shard_range(total: int, rank: int, world: int):
    """(offset, count) of rank's contiguous block of `total` chains."""
    if world < 1 or not 0 <= rank < world or total < world:
        raise ValueError("need 0 <= rank < world <= total")
    base, rem = divmod(total, world)
    return rank * base + min(rank, rem), base + (1 if rank < rem else 0)


def minloc(f: float, index: int, x, group=None):
    """All ranks: the lowest (f, global index) over the ranks and its state x."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    key = float(f) if not math.isnan(f) else math.inf
    mine = torch.tensor([key, float(index), 0.0 if not math.isnan(f) else 1.0], dtype=torch.float64)
    every = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    rows = [(e[2].item(), e[0].item(), e[1].item(), r) for r, e in enumerate(every)]
    nan_flag, fbest, ibest, owner = min(rows)
    xt = torch.as_tensor(np.asarray(x, np.float64)).clone()
    src = dist.get_global_rank(group, owner) if group is not None else owner
    dist.broadcast(xt, src=src, group=group)
    return (math.nan if nan_flag else fbest), int(ibest), xt.numpy()


class HandleShard:
    """A single-problem solver handle (sa.create) as one shard of a sharded run."""

    def __init__(self, handle, offset: int):
        self.h = handle
        self.offset = int(offset)
        handle.set_chain_offset(self.offset)

    def run_level(self):
        self.h.run(1)
        local = int(self.h.level_log()["argmin"][-1])
        x, f = self.h.restart_point()
        return f, self.offset + local, x

    def set_restart(self, x, f: float, index: int):
        self.h.set_restart(x, f, index)


def run_sharded(shard, levels: int, group=None):
    """Run `levels` levels of `shard` with an exchange after each one.  Returns the
    global argmin and value of every level and the incumbent (the lowest of them)."""
    argmins, f_level = [], []
    f_inc, x_inc = math.inf, None
    for level in range(levels):
        f, index, x = shard.run_level()
        try:
            F, I, X = minloc(f, index, x, group)
        except RuntimeError as err:  # a peer stopped or the process group timed out
            raise ShardError(f"exchange after level {level} failed: {err}") from err
        if math.isnan(F):
            raise ShardError(f"no finite state after level {level}")
        shard.set_restart(X, F, I)
        argmins.append(I)
        f_level.append(F)
        if F < f_inc:
            f_inc, x_inc = F, X.copy()
    return {"argmin": np.array(argmins, np.int64), "f_level": np.array(f_level), "f_inc": f_inc, "x_inc": x_inc}
