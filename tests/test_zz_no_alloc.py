"""The allocation-free MotionValidation entry point.

mv_validate_noalloc serves callers that cannot allocate device memory while
validating (latency-bounded control loops, where cudaMalloc / cudaFree may
block or synchronize the device, and applications whose device memory is
budgeted by their own allocator).  Its scratch is a static device array
shared by all calls, so the test runs it twice in a row on different batches
and checks each result against mv_validate on the same inputs.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
from __future__ import annotations

import os
import time

import numpy as np
import pytest

from paper_2604_23960_gb300 import mrv
from paper_2604_23960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ref_and_noalloc(ctx, ba):
    import torch
    ref = ctx.mv_validate(ba)                      # existing entry point
    out = torch.full((ba.n_queries,), 7, dtype=torch.uint8, device="cuda")
    mrv.mv_validate_noalloc(ctx.h, ba.struct(mrv.MRV_CHECK_ENV), out)
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_matches_mv_validate_twice():
    ctx = mrv.Context(0)
    arms = ctx.bind(W.make_cage_mv(1500, query_seed=611)).to("cuda")
    discs = ctx.bind(W.make_plain_discs(700, query_seed=612)).to("cuda")
    team16 = ctx.bind(W.make_cage16_mv(300, query_seed=613)).to("cuda")   # the large-team instance
    for ba in (arms, discs, team16, arms):         # back-to-back calls share the scratch
        ref, got = _ref_and_noalloc(ctx, ba)
        np.testing.assert_array_equal(got, ref)
    ctx.close()


def test_noalloc_allocates_nothing():
    """On a fresh context (its scratch arena never allocated), the library's
    next device allocation is made to fail; the allocation-free call still
    succeeds, and the mv_validate after it fails with MRV_ERR_OOM, which
    shows the injected failure was still armed during the first call.  The
    statistics then describe the allocation-free call."""
    import torch
    ctx = mrv.Context(0)
    try:
        ba = ctx.bind(W.make_cage_mv(800, query_seed=614)).to("cuda")   # uploads allocate here
        out = torch.full((ba.n_queries,), 7, dtype=torch.uint8, device="cuda")
        os.environ["MRV_FAULT_INJECT_ALLOC"] = f"noalloc-{os.getpid()}-{time.monotonic_ns()}"
        try:
            mrv.mv_validate_noalloc(ctx.h, ba.struct(mrv.MRV_CHECK_ENV), out)
            st = ctx.stats()
            with pytest.raises(mrv.MrvError) as e:
                ctx.mv_validate(ba)
            assert e.value.code == -2
        finally:
            del os.environ["MRV_FAULT_INJECT_ALLOC"]
        ref = ctx.mv_validate(ba).cpu().numpy()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        assert st["n_valid"] == int(ref.sum())
        assert 0 < st["states_checked"] <= st["states_available"]
        assert st["work_items"] > 0
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    ctx = mrv.Context(0)
    ba = ctx.bind(W.make_plain_discs(mrv.MRV_NOALLOC_MAX_QUERIES + 1)).to("cuda")
    import torch
    out = torch.empty(ba.n_queries, dtype=torch.uint8, device="cuda")
    with pytest.raises(mrv.MrvError) as e:
        mrv.mv_validate_noalloc(ctx.h, ba.struct(mrv.MRV_CHECK_ENV), out)
    assert e.value.code == -7
    ctx.close()
