"""Serving: every request's results are the same when it runs alone
(mrv_run on the context) and when it runs mixed with concurrent requests
from many client threads through the continuous-batching server."""
from __future__ import annotations

import threading

import numpy as np
import pytest

from paper_2604_23960_gb300 import mrv
from paper_2604_23960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_alone_equals_mixed():
    ctx = mrv.Context(0)
    models, envs, fams = W.make_serving_families(600, seed=11)
    rids = [ctx.upload_model(m) for m in models]
    eids = [ctx.upload_env(e) for e in envs]
    rng = np.random.default_rng(12)
    reqs = []
    for k in range(48):
        f = fams[k % 4]
        ba = ctx.bind(f, rids, eids)
        n = int(rng.integers(1, 120))
        q0 = int(rng.integers(0, f.batch.n_queries - n))
        reqs.append(mrv.slice_batch(ba, q0, q0 + n))
    alone = [ctx.run(r) for r in reqs]
    srv = mrv.Server(ctx, n_streams=4, device_budget_bytes=256 << 20, max_batch_queries=400, max_pending=1000)
    got = [None] * len(reqs)

    def client(ids):
        for i in ids:
            t = srv.submit(reqs[i])
            got[i] = srv.wait(t, reqs[i].n_queries, timeout_ms=60000)

    th = [threading.Thread(target=client, args=(list(range(c, len(reqs), 8)),)) for c in range(8)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st = srv.stats()
    srv.close()
    for r, (va, ca), (vm, cm) in zip(reqs, alone, got):
        kind = r.a["q_kind"]
        np.testing.assert_array_equal(va[kind == 0], vm[kind == 0])
        np.testing.assert_array_equal(ca[kind == 1], cm[kind == 1])
    assert st["completed"] == len(reqs) and st["submitted"] == len(reqs)
    assert st["micro_batches"] >= 1
    ctx.close()


def test_admission_rejects_oversized_request():
    ctx = mrv.Context(0)
    w = W.make_plain_discs(2000)
    ba = ctx.bind(w)
    ba.a["q_kind"] = np.zeros(w.batch.n_queries, np.uint8)
    srv = mrv.Server(ctx, n_streams=1, device_budget_bytes=4096, max_batch_queries=100, max_pending=4)
    with pytest.raises(mrv.MrvError) as e:
        srv.submit(ba)
    assert e.value.code == -6
    assert srv.stats()["rejected"] == 1
    srv.close()
    ctx.close()


def test_wait_times_out_and_unknown_ticket():
    ctx = mrv.Context(0)
    srv = mrv.Server(ctx, n_streams=1)
    with pytest.raises(mrv.MrvError) as e:
        srv.wait(12345, 1, timeout_ms=10)
    assert e.value.code == -3
    srv.close()
    ctx.close()


def test_no_allocation_while_serving():
    """Each stream's device arena and pinned staging are sized when the server
    is created, so serving requests that fit a micro-batch allocates nothing:
    with the library's next device allocation made to fail, every request
    still completes with its alone result, and the allocation failure is
    still armed afterwards.  The budget in force is clamped to the device."""
    import os
    import time
    ctx = mrv.Context(0)
    models, envs, fams = W.make_serving_families(400, seed=21)
    rids = [ctx.upload_model(m) for m in models]
    eids = [ctx.upload_env(e) for e in envs]
    rng = np.random.default_rng(22)
    reqs = []
    for k in range(32):
        f = fams[k % 4]
        ba = ctx.bind(f, rids, eids)
        n = int(rng.integers(1, 100))
        q0 = int(rng.integers(0, f.batch.n_queries - n))
        reqs.append(mrv.slice_batch(ba, q0, q0 + n))
    alone = [ctx.run(r) for r in reqs]
    srv = mrv.Server(ctx, n_streams=3, device_budget_bytes=1 << 60, max_batch_queries=512, max_pending=1000)
    st0 = srv.stats()
    assert 0 < st0["device_budget_bytes"] < (1 << 60) and st0["presized_queries"] == 512
    os.environ["MRV_FAULT_INJECT_ALLOC"] = f"serve-{os.getpid()}-{time.monotonic_ns()}"
    try:
        got = [None] * len(reqs)

        def client(ids):
            for i in ids:
                t = srv.submit(reqs[i])
                got[i] = srv.wait(t, reqs[i].n_queries, timeout_ms=60000)

        th = [threading.Thread(target=client, args=(list(range(c, len(reqs), 6)),)) for c in range(6)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        with pytest.raises(mrv.MrvError) as e:
            ctx.upload_model(models[0])          # the injected failure was still armed
        assert e.value.code == -2
    finally:
        del os.environ["MRV_FAULT_INJECT_ALLOC"]
    srv.close()
    for r, (va, ca), (vm, cm) in zip(reqs, alone, got):
        kind = r.a["q_kind"]
        np.testing.assert_array_equal(va[kind == 0], vm[kind == 0])
        np.testing.assert_array_equal(ca[kind == 1], cm[kind == 1])
    ctx.close()
