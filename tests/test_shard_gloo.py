"""Sharded chains with the per-level exchange, as gloo ranks on the CPU.

Each rank runs its block of chains with the oracle (the logic under test is the
exchange and the restart, not the sweep), exchanges through
paper_2408_00018_gb300.shard, and must reproduce the unsharded oracle run bit
for bit.  Failure detection: a rank that exits, or that never joins an
exchange, makes the other rank's next exchange raise ShardError within the
process group's timeout.
"""
import datetime
import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2408_00018_gb300 import inputs
from paper_2408_00018_gb300.shard import ShardError, run_sharded, shard_range

CFG = dict(cost="schwefel", n=3, C=301, L=40, K=5, T0=50.0, rho=0.8, seed=12)


class OracleShard:
    """A block of the global chains run by the oracle, one level at a time."""

    def __init__(self, p, offset, count):
        self.p, self.offset, self.count = p, offset, count
        self.level, self.x_start = 0, None

    def run_level(self):
        r = self.p.level_chains(self.level, self.offset, self.offset + self.count, x_start=self.x_start, want_x=True)
        F = np.where(np.isnan(r["F"]), np.inf, r["F"])
        i = int(np.argmin(F))
        return float(r["F"][i]), self.offset + i, r["X"][i]

    def set_restart(self, x, f, index):
        self.x_start = np.array(x, np.float64)
        self.level += 1


def _problem():
    lo, hi = inputs.box(CFG["cost"], CFG["n"])
    return oracle.Problem(CFG["cost"], CFG["n"], lo, hi, chains=CFG["C"], L=CFG["L"], T0=CFG["T0"], rho=CFG["rho"],
                          seed=CFG["seed"], mode=0, threads=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=4))
    off, cnt = shard_range(CFG["C"], rank, world)
    shard = OracleShard(_problem(), off, cnt)
    result = "ok"
    try:
        if mode == "ok":
            r = run_sharded(shard, CFG["K"])
            np.savez(os.path.join(outdir, f"r{rank}.npz"), argmin=r["argmin"], f_level=r["f_level"], f_inc=r["f_inc"],
                     x_inc=r["x_inc"])
        elif rank == 1 and mode == "exit":
            run_sharded(shard, 1)  # one level with the others, then the process ends
            os._exit(0)
        elif rank == 1 and mode == "silent":
            import time
            run_sharded(shard, 1)
            time.sleep(8)  # never joins the next exchange
        else:
            run_sharded(shard, CFG["K"])
    except ShardError as e:
        result = "ShardError: " + str(e)
    with open(os.path.join(outdir, f"status{rank}.txt"), "w") as fh:
        fh.write(result)
    if mode == "ok":
        dist.destroy_process_group()
    os._exit(0)


def _spawn(mode, tmp_path, world=2):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.start_processes(_worker, args=(world, port, mode, str(tmp_path)), nprocs=world, join=False,
                             start_method="spawn")
    import time
    deadline = time.monotonic() + 120
    while not ctx.join(timeout=5):  # join returns once any process ends: wait for all of them
        if time.monotonic() > deadline:
            for proc in ctx.processes:
                proc.kill()
            break
    return {r: (tmp_path / f"status{r}.txt").read_text() if (tmp_path / f"status{r}.txt").exists() else None
            for r in range(world)}


def test_shard_range_partitions():
    for total, world in [(10, 3), (301, 2), (8, 8), (1 << 20, 7)]:
        blocks = [shard_range(total, r, world) for r in range(world)]
        assert blocks[0][0] == 0 and sum(c for _, c in blocks) == total
        assert all(blocks[r][0] + blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
    with pytest.raises(ValueError):
        shard_range(3, 0, 4)


def test_two_ranks_reproduce_the_unsharded_run(tmp_path):
    status = _spawn("ok", tmp_path)
    assert status == {0: "ok", 1: "ok"}, status
    ref = _problem().run(CFG["K"])
    for r in range(2):
        d = np.load(tmp_path / f"r{r}.npz")
        assert np.array_equal(d["argmin"], ref["argmin"])
        assert np.array_equal(d["f_level"], ref["f_level"])
        assert float(d["f_inc"]) == ref["f_inc"] and np.array_equal(d["x_inc"], ref["x_inc"])


@pytest.mark.parametrize("mode", ["exit", "silent"])
def test_a_stopped_rank_is_detected_at_the_next_exchange(tmp_path, mode):
    status = _spawn(mode, tmp_path)
    assert status[0] is not None and status[0].startswith("ShardError"), status
    assert "after level 1" in status[0]
