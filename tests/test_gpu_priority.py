"""MV of prioritized planning (MRV_PRIORITY, Sec. IV-C) on the GPU against the
oracle's prioritized MV: random point and chain robots (2-4 per query), three
discs (the lane-per-state kernel), the cage edge checks at small and full size,
every code path (dense, broadphase, one launch per query, hierarchical and
linear orders), the minimum clearance of exhaustive runs, and mixed mrv_run
batches (FFC queries ignore the flag)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_23960_gb300 import mrv
from paper_2604_23960_gb300 import workloads as W
from tests import parity as PA
from tests.tiny import tiny_workload

pytestmark = pytest.mark.gpu

PRIO = mrv.MRV_PRIORITY


@pytest.fixture(scope="module")
def ctx():
    c = mrv.Context(0)
    yield c
    c.close()


def _np(x):
    return x.cpu().numpy() if isinstance(x, torch.Tensor) else np.asarray(x)


@pytest.mark.parametrize("seed", range(4))
def test_tiny_priority(ctx, seed):
    w = tiny_workload(900 + seed, n_queries=40, timed=bool(seed % 2), max_robots=4)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    for ce in (True, False):
        v = ctx.mv_validate(ba, check_env=ce, flags=PRIO)
        PA.check_mv(o, v, check_env=ce, priority=True)
        for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_PER_QUERY_LAUNCH, mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR):
            np.testing.assert_array_equal(ctx.mv_validate(ba, check_env=ce, flags=PRIO | fl), v)
        v2, mc = ctx.mv_validate(ba, check_env=ce, exhaustive=True, min_clearance=True, flags=PRIO)
        np.testing.assert_array_equal(v2, v)
        ref = o.mv_min_clearance(check_env=ce, priority=True)
        fin = np.isfinite(ref)
        np.testing.assert_array_equal(np.isfinite(mc), fin)
        np.testing.assert_allclose(mc[fin], ref[fin], atol=PA.CLR_TOL, rtol=0)
        # the full MV is never valid where the prioritized one is not
        full = ctx.mv_validate(ba, check_env=ce)
        dec = np.abs(o.mv_min_clearance(check_env=ce)) > PA.MARGIN
        assert not np.any(full.astype(bool) & ~v.astype(bool) & dec)


def test_three_discs_priority(ctx):
    """Three discs per query in the box world (point robots: one lane per
    state): obstacles and meetings count only when disc 0 takes part."""
    rng = np.random.default_rng(41)
    disc = W.disc_robot(0.25)
    env = W.world_boxes(101)
    bb = W.BatchBuilder(2, True)
    for _ in range(300):
        T = int(rng.integers(5, 120))
        paths = [np.array([rng.uniform(0, 10, 2), rng.uniform(0, 10, 2)], np.float32) for _ in range(3)]
        bb.add([0, 0, 0], paths, [[T]] * 3, 0, 0)
    w = W.Workload("discs3", [disc], [env], bb.build(0.05), env=0, check_env=True)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    for ce in (True, False):
        v = ctx.mv_validate(ba, check_env=ce, flags=PRIO)
        n, und = PA.check_mv(o, v, check_env=ce, priority=True)
        assert und < 10
        np.testing.assert_array_equal(ctx.mv_validate(ba, check_env=ce, flags=PRIO | mrv.MRV_PER_QUERY_LAUNCH), v)
    full = ctx.mv_validate(ba)
    prio = ctx.mv_validate(ba, flags=PRIO)
    assert prio.sum() > full.sum()   # meetings of discs 1 and 2 no longer count


def test_cage_priority_small(ctx):
    w = W.make_cage_priority(300)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba, flags=PRIO))
    PA.check_mv(o, v, priority=True)
    assert 0.1 < v.mean() < 0.6
    for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR):
        np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=PRIO | fl)), v)
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True, flags=PRIO)
    np.testing.assert_array_equal(_np(v2), v)
    ref = o.mv_min_clearance(threads=PA.THREADS, priority=True)
    np.testing.assert_allclose(_np(mc), ref, atol=PA.CLR_TOL, rtol=0)
    st = ctx.stats()
    assert st["states_checked"] == st["states_available"]
    # the prioritized check runs a quarter of the robot-robot pairs and a
    # quarter of the obstacle and self tests of the full MV
    ctx.mv_validate(ba, exhaustive=True, flags=PRIO | mrv.MRV_NO_BROADPHASE)
    st_p = ctx.stats()
    ctx.mv_validate(ba, exhaustive=True, flags=mrv.MRV_NO_BROADPHASE)
    st_f = ctx.stats()
    assert st_p["sphere_tests"] == st_p["sphere_tests_available"]
    per_state_p = 64 * 192 + 64 * 52 + 1342
    per_state_f = 6 * 64 * 64 + 256 * 52 + 4 * 1342
    assert st_p["sphere_tests"] * per_state_f == st_f["sphere_tests"] * per_state_p


def test_full_cage_priority_10k(ctx):
    """The benchmark's size and launch (device batch): all 10,000 edges
    against the oracle."""
    w = W.make_cage_priority(10000)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba, flags=PRIO))
    n, _ = PA.check_mv(o, v, priority=True)
    assert n == 10000


def test_mixed_run_ignores_priority_for_ffc(ctx):
    w = tiny_workload(950, n_queries=60, timed=True, max_robots=4)
    kind = np.random.default_rng(3).integers(0, 2, w.batch.n_queries).astype(np.uint8)
    w.batch.q_kind = kind
    o = O.Oracle(w)
    ba = ctx.bind(w)
    v, c = ctx.run(ba, flags=PRIO)
    v0, c0 = ctx.run(ba)
    ffq = kind == 1
    np.testing.assert_array_equal(c[ffq], c0[ffq])
    mvq = np.nonzero(kind == 0)[0]
    PA.check_mv(o, v[mvq], idx=mvq, priority=True)
