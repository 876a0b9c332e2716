"""Multi-rank host path on the CPU: two gloo ranks split a batch by cost,
validate their shards (with the oracle: no GPU here) and gather the results;
rank 0's assembled answer equals the single-process one."""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_23960_gb300 import multi
from paper_2604_23960_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ret):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    w = W.make_ragged_teams(60, seed=31, len_range=(8, 24))
    b = w.batch
    shards = multi.shard_by_cost(multi.query_costs(b.q_robot_off, b.slot_wp_off, b.seg_steps), world)
    mine = shards[rank]
    o = O.Oracle(w)
    ffc = o.ffc(mine)
    full = multi.gather_results(mine, ffc, b.n_queries, world, rank)
    if rank == 0:
        ret["full"] = full
        ret["ref"] = o.ffc()
        ret["sizes"] = [len(s) for s in shards]
    dist.destroy_process_group()


def test_two_ranks_gloo():
    mp_ctx = mp.get_context("spawn")
    mgr = mp_ctx.Manager()
    ret = mgr.dict()
    port = _free_port()
    procs = [mp_ctx.Process(target=_worker, args=(r, 2, port, ret)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    np.testing.assert_array_equal(ret["full"], ret["ref"])
    assert sum(ret["sizes"]) == 60 and min(ret["sizes"]) > 0


def test_partition_is_balanced_and_complete():
    rng = np.random.default_rng(3)
    costs = rng.lognormal(0, 1.5, 1000)
    for world in (1, 2, 3, 8):
        sh = multi.shard_by_cost(costs, world)
        allq = np.concatenate(sh)
        assert sorted(allq) == list(range(1000))
        loads = [costs[s].sum() for s in sh]
        assert max(loads) - min(loads) <= costs.max() + 1e-9
        assert [list(s) for s in multi.shard_by_cost(costs, world)] == [list(s) for s in sh]
