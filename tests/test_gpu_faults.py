"""Failure detection without a GPU fault.

* a kernel budget that runs out makes the call return MRV_ERR_TIMEOUT (the
  persistent kernel stops taking work items; nothing spins or traps), and the
  context stays usable;
* an injected device-allocation failure (host side) is reported as
  MRV_ERR_OOM and the next call succeeds;
* malformed batches are rejected with status codes, the context stays usable;
* a client that abandons a request does not keep the server from shutting
  down.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_2604_23960_gb300 import mrv
from paper_2604_23960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = mrv.Context(0)
    yield c
    c.close()


def test_kernel_budget_timeout_then_recovery(ctx):
    w = W.make_cage_ffc(20000, query_seed=41)
    ba = ctx.bind(w).to("cuda")
    ref = ctx.ffc_find(ba).cpu().numpy()
    mrv.mrv_set_limits(ctx.h, 1e-4)          # 0.1 us: runs out at once
    try:
        with pytest.raises(mrv.MrvError) as e:
            ctx.ffc_find(ba)
        assert e.value.code == -5
    finally:
        mrv.mrv_set_limits(ctx.h, 0.0)
    np.testing.assert_array_equal(ctx.ffc_find(ba).cpu().numpy(), ref)
    mrv.mrv_set_limits(ctx.h, 60000.0)       # a generous bound changes nothing
    np.testing.assert_array_equal(ctx.ffc_find(ba).cpu().numpy(), ref)
    mrv.mrv_set_limits(ctx.h, 0.0)


def test_injected_allocation_failure(ctx):
    w = W.make_plain_discs(50)
    os.environ["MRV_FAULT_INJECT_ALLOC"] = "upload-1"
    try:
        with pytest.raises(mrv.MrvError) as e:
            ctx.upload_model(w.models[0])
        assert e.value.code == -2
    finally:
        del os.environ["MRV_FAULT_INJECT_ALLOC"]
    fresh = mrv.Context(0)                      # its scratch arena is still empty
    try:
        ba = fresh.bind(w)
        os.environ["MRV_FAULT_INJECT_ALLOC"] = "scratch-1"
        try:
            with pytest.raises(mrv.MrvError) as e:
                fresh.mv_validate(ba)           # the first call allocates the arena
            assert e.value.code == -2
        finally:
            del os.environ["MRV_FAULT_INJECT_ALLOC"]
        assert fresh.mv_validate(ba).shape == (50,)
    finally:
        fresh.close()


def test_malformed_batches_keep_context_usable(ctx):
    w = W.make_plain_discs(10)
    ba = ctx.bind(w)
    bad = dict(ba.a)
    bad["slot_wp_off"] = ba.a["slot_wp_off"].copy()
    bad["slot_wp_off"][-1] += 5                 # offsets past the waypoint array
    b2 = mrv.BatchArrays(bad, ba.n_queries, ba.n_slots, ba.n_waypoints, ba.wp_stride, ba.resolution, ba.env_id, False)
    with pytest.raises(mrv.MrvError) as e:
        ctx.mv_validate(b2)
    assert e.value.code == -1
    b3 = mrv.BatchArrays(dict(ba.a), ba.n_queries, ba.n_slots, ba.n_waypoints, ba.wp_stride, -1.0, ba.env_id, False)
    with pytest.raises(mrv.MrvError):
        ctx.mv_validate(b3)                     # start/goal form needs a positive resolution
    b4 = mrv.BatchArrays(dict(ba.a), ba.n_queries, ba.n_slots, ba.n_waypoints, ba.wp_stride, ba.resolution,
                         12345, False)
    with pytest.raises(mrv.MrvError) as e:
        ctx.mv_validate(b4)                     # unknown env id
    assert e.value.code == -3
    assert ctx.mv_validate(ba).shape == (10,)


def test_abandoned_request_does_not_block_shutdown(ctx):
    models, envs, fams = W.make_serving_families(200, seed=5)
    rids = [ctx.upload_model(m) for m in models]
    eids = [ctx.upload_env(e) for e in envs]
    ba = ctx.bind(fams[1], rids, eids)
    srv = mrv.Server(ctx, n_streams=2, max_pending=2)
    t1 = srv.submit(mrv.slice_batch(ba, 0, 50))
    srv.submit(mrv.slice_batch(ba, 50, 100))    # never waited for
    v, c = srv.wait(t1, 50, timeout_ms=60000)
    assert v.shape == (50,)
    # a full queue refuses with MRV_ERR_BUSY instead of blocking
    codes = []
    for k in range(50):
        try:
            srv.submit(mrv.slice_batch(ba, 0, 200))
        except mrv.MrvError as e:
            codes.append(e.code)
    assert codes == [] or set(codes) == {-6}
    srv.close()                                  # returns: pending work drains, nothing hangs
