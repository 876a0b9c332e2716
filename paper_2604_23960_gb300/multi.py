"""Multi-GPU host logic: queries are independent, so N GPUs run replicas.

A batch is split across ranks by estimated cost (longest-processing-time
greedy on robot pairs x states), every rank validates its shard on its own
GPU through the C ABI (run_sharded) with no collective on the data path, and
the per-query results are gathered on the host.  Every rank computes the
same partition from the same arrays, so nothing but results crosses process
boundaries.
"""
from __future__ import annotations

import heapq
from typing import List

import numpy as np


def query_costs(q_robot_off: np.ndarray, slot_wp_off: np.ndarray, seg_steps=None) -> np.ndarray:
    """Relative cost per query: (robot pairs + 1) x (states, from the first
    slot's step counts in the timed form, 1 otherwise)."""
    n = np.diff(q_robot_off).astype(np.int64)
    pairs = n * (n - 1) // 2 + 1
    if seg_steps is None:
        return pairs.astype(np.float64)
    first = q_robot_off[:-1]
    w0, w1 = slot_wp_off[first], slot_wp_off[first + 1]
    csum = np.concatenate([[0], np.cumsum(seg_steps.astype(np.int64))])
    states = csum[w1 - 1] - csum[w0] + 1
    return (pairs * states).astype(np.float64)


def shard_by_cost(costs: np.ndarray, world: int) -> List[np.ndarray]:
    """Greedy LPT partition of query indices into `world` shards (sorted
    indices per shard); deterministic: ties go to the lower rank / index."""
    order = np.lexsort((np.arange(len(costs)), -costs))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for q in order:
        load, r = heapq.heappop(heap)
        out[r].append(int(q))
        heapq.heappush(heap, (load + float(costs[q]), r))
    return [np.array(sorted(s), dtype=np.int64) for s in out]


def gather_results(local_idx: np.ndarray, local_out: np.ndarray, n_total: int, world: int, rank: int,
                   group=None):
    """Collects every rank's (indices, results) on rank 0 (torch.distributed,
    any backend; `group` may name a host-side gloo group so that the GPU
    ranks' NCCL communicator carries no data); returns the assembled array
    on rank 0 and None elsewhere."""
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object((np.asarray(local_idx), np.asarray(local_out)), parts, dst=0, group=group)
    if rank != 0:
        return None
    shape = (n_total,) + tuple(np.asarray(local_out).shape[1:])
    full = np.zeros(shape, dtype=np.asarray(local_out).dtype)
    seen = np.zeros(n_total, dtype=bool)
    for idx, out in parts:
        full[idx] = out
        seen[idx] = True
    if not seen.all():
        raise RuntimeError("some queries were not validated by any rank")
    return full


def take_queries(ba, idx):
    """The queries `idx` (sorted) of a host batch (mrv.BatchArrays with numpy
    arrays) as a new host batch: the CSR arrays are gathered, slot and
    waypoint offsets renumbered; uploaded robot and env ids are kept."""
    from . import mrv
    a = ba.a
    idx = np.asarray(idx, np.int64)
    qo = np.asarray(a["q_robot_off"], np.int64)
    so = np.asarray(a["slot_wp_off"], np.int64)
    n_rob = qo[idx + 1] - qo[idx]
    new_qo = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(n_rob, out=new_qo[1:])
    slots = np.repeat(qo[idx], n_rob) + (np.arange(new_qo[-1]) - np.repeat(new_qo[:-1], n_rob))
    n_wp = so[slots + 1] - so[slots]
    new_so = np.zeros(len(slots) + 1, np.int64)
    np.cumsum(n_wp, out=new_so[1:])
    wps = np.repeat(so[slots], n_wp) + (np.arange(new_so[-1]) - np.repeat(new_so[:-1], n_wp))
    out = {
        "q_robot_off": new_qo.astype(np.int32),
        "slot_robot_id": np.ascontiguousarray(np.asarray(a["slot_robot_id"])[slots], np.int32),
        "slot_wp_off": new_so.astype(np.int32),
        "waypoints": np.ascontiguousarray(np.asarray(a["waypoints"])[wps], np.float32),
        "seg_steps": None if a.get("seg_steps") is None else np.ascontiguousarray(np.asarray(a["seg_steps"])[wps],
                                                                                 np.int32),
        "q_env_id": None if a.get("q_env_id") is None else np.ascontiguousarray(np.asarray(a["q_env_id"])[idx],
                                                                               np.int32),
        "q_kind": None if a.get("q_kind") is None else np.ascontiguousarray(np.asarray(a["q_kind"])[idx], np.uint8),
    }
    return mrv.BatchArrays(out, len(idx), len(slots), int(new_so[-1]), ba.wp_stride, ba.resolution, ba.env_id,
                           False)


def shard_of(ba, world: int, rank: int) -> np.ndarray:
    """This rank's queries of a host batch under the cost partition (every
    rank computes the same partition from the same arrays)."""
    a = ba.a
    costs = query_costs(np.asarray(a["q_robot_off"]), np.asarray(a["slot_wp_off"]),
                        None if a.get("seg_steps") is None else np.asarray(a["seg_steps"]))
    return shard_by_cost(costs, world)[rank]


def run_sharded(ctx, ba, world: int, rank: int, check_env: bool = True, group=None):
    """Validates one host batch split across `world` ranks: this rank runs its
    cost shard through mrv_run on its own GPU (ctx), and the per-query
    results are gathered on rank 0.  Returns (valid, conflicts) for the whole
    batch on rank 0 (each meaningful where the query's kind selects it, as
    for mrv_run) and None elsewhere.  No collective touches the device."""
    mine = shard_of(ba, world, rank)
    sub = take_queries(ba, mine)
    v, c = ctx.run(sub, check_env=check_env)
    v = v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)
    c = c.cpu().numpy() if hasattr(c, "cpu") else np.asarray(c)
    full_v = gather_results(mine, v, ba.n_queries, world, rank, group=group)
    full_c = gather_results(mine, c, ba.n_queries, world, rank, group=group)
    return None if rank != 0 else (full_v, full_c)
