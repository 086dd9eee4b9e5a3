"""Sharded solvers on one GPU: two handles own the two halves of the global
chains (sa_set_chain_offset) and exchange their level minima on the host
(sa_restart_point / sa_set_restart).  The levels must be those of the
unsharded run, bit for bit, on the FP64, FP32 and rotated paths.  (The
handles run one after the other; no kernel waits on another shard.)"""
import math

import numpy as np
import pytest

from paper_2408_00018_gb300 import inputs
from paper_2408_00018_gb300.shard import HandleShard, shard_range

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_00018_gb300 import sa as sa_mod
    return sa_mod


@pytest.mark.parametrize("cost,n,C,prec", [("schwefel", 2, 1001, "fp64"), ("rastrigin", 24, 3000, "fp32"),
                                           ("rot_schwefel", 40, 700, "fp32")])
def test_two_shards_reproduce_the_unsharded_run(sa, cost, n, C, prec):
    L, K = 60, 5
    lo, hi = inputs.box(cost, n)
    Q = inputs.rotation(n, 1) if cost.startswith("rot") else None
    sch = sa.Schedule(T0=20.0, rho=0.8, levels=K, precision=prec)
    full = sa.create(cost, lo, hi, n, C, L, sch, seed=6, Q=Q)
    full.run()
    ref = full.level_log()
    _, f_ref, _ = full.best()
    shards = []
    for r in range(2):
        off, cnt = shard_range(C, r, 2)
        shards.append(HandleShard(sa.create(cost, lo, hi, n, cnt, L, sch, seed=6, Q=Q), off))
    for level in range(K):
        results = [s.run_level() for s in shards]
        f, i, x = min(results, key=lambda t: (math.isnan(t[0]), t[0], t[1]))
        for s in shards:
            s.set_restart(x, f, i)
        assert i == ref["argmin"][level] and f == ref["f_level"][level], (level, i, f)
    for s in shards:
        assert np.array_equal(s.h.level_log()["argmin"], ref["argmin"])
        assert s.h.best()[1] == f_ref
