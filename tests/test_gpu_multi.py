"""The multi-rank path through the C ABI: two gloo ranks (both on GPU 0, each
with its own context and stream; their kernels never wait on one another)
split one mixed batch by cost with multi.run_sharded, validate their shards
with mrv_run and gather the results on rank 0; the gathered answer equals
the single-process answer of the same batch."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_2604_23960_gb300 import multi
from paper_2604_23960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ret):
    import torch
    import torch.distributed as dist
    from paper_2604_23960_gb300 import mrv
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    ctx = mrv.Context(0)
    w = W.make_ragged_teams(4000, seed=83)
    ba = ctx.bind(w)
    res = multi.run_sharded(ctx, ba, world, rank)
    if rank == 0:
        ret["valid"], ret["conf"] = res
        ret["shard"] = len(multi.shard_of(ba, world, 0))
    ctx.close()
    dist.destroy_process_group()


def test_two_ranks_sharded_cuda_path():
    import torch.multiprocessing as mp
    from paper_2604_23960_gb300 import mrv
    mp_ctx = mp.get_context("spawn")
    mgr = mp_ctx.Manager()
    ret = mgr.dict()
    port = _free_port()
    procs = [mp_ctx.Process(target=_worker, args=(r, 2, port, ret)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    w = W.make_ragged_teams(4000, seed=83)
    ctx = mrv.Context(0)
    v, c = ctx.run(ctx.bind(w))
    ctx.close()
    k = w.batch.q_kind
    np.testing.assert_array_equal(ret["valid"][k == 0], v[k == 0])
    np.testing.assert_array_equal(ret["conf"][k == 1], c[k == 1])
    assert 0 < ret["shard"] < 4000
