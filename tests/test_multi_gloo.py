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


def test_take_queries_equals_subset():
    """The vectorised CSR gather of run_sharded's shards equals the
    query-by-query subset of the workload module."""
    from paper_2604_23960_gb300 import mrv
    for w in (W.make_ragged_teams(300, seed=9), W.make_cage_mv(50)):
        b = w.batch
        arrays = {"q_robot_off": b.q_robot_off.astype(np.int32), "slot_robot_id": b.slot_robot.astype(np.int32),
                  "slot_wp_off": b.slot_wp_off.astype(np.int32), "waypoints": b.waypoints,
                  "seg_steps": b.seg_steps, "q_env_id": b.q_env, "q_kind": b.q_kind}
        ba = mrv.BatchArrays(arrays, b.n_queries, int(b.q_robot_off[-1]), int(b.slot_wp_off[-1]), b.wp_stride,
                             b.resolution, 0, False)
        idx = np.sort(np.random.default_rng(1).choice(b.n_queries, 17, replace=False))
        t = multi.take_queries(ba, idx)
        ws = W.subset(w, idx).batch
        for k, ref in (("q_robot_off", ws.q_robot_off), ("slot_robot_id", ws.slot_robot),
                       ("slot_wp_off", ws.slot_wp_off), ("waypoints", ws.waypoints), ("seg_steps", ws.seg_steps),
                       ("q_kind", ws.q_kind)):
            if ref is None:
                assert t.a[k] is None
            else:
                np.testing.assert_array_equal(np.asarray(t.a[k]), np.asarray(ref))
        assert (t.n_queries, t.n_slots, t.n_waypoints) == (17, int(ws.q_robot_off[-1]), int(ws.slot_wp_off[-1]))
