"""Multi-GPU host logic: queries are independent, so N GPUs run replicas.

A batch is split across ranks by estimated cost (longest-processing-time
greedy on robot pairs x states), every rank validates its shard on its own
GPU with no collective on the data path, and the per-query results are
gathered on the host.  Every rank computes the same partition from the same
arrays, so nothing but results crosses process boundaries.
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


def gather_results(local_idx: np.ndarray, local_out: np.ndarray, n_total: int, world: int, rank: int):
    """Collects every rank's (indices, results) on rank 0 (torch.distributed,
    any backend); returns the assembled array on rank 0 and None elsewhere."""
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object((np.asarray(local_idx), np.asarray(local_out)), parts, dst=0)
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
