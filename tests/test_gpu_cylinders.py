"""Cylinder obstacles (the Cage scenario's obstacle kind, Sec. V-A) on the GPU
against the oracle: random robots in scenes with cylinders (every code path,
minimum clearance, the prioritized variant), discs past vertical cylinders
(the lane-per-state kernel), the floor- and ceiling-mounted 8-arm team in the
cylinder cage at small and at full size, the per-sphere clearance diagnostic,
and the upload's argument checks."""
from __future__ import annotations

import copy

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_23960_gb300 import mrv
from paper_2604_23960_gb300 import workloads as W
from tests import parity as PA
from tests.tiny import tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = mrv.Context(0)
    yield c
    c.close()


def _np(x):
    return x.cpu().numpy() if isinstance(x, torch.Tensor) else np.asarray(x)


@pytest.mark.parametrize("seed", range(4))
def test_tiny_cylinders(ctx, seed):
    w = tiny_workload(1400 + seed, n_queries=40, timed=bool(seed % 2), max_robots=4, cylinders=6)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    v = ctx.mv_validate(ba)
    PA.check_mv(o, v)
    for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_PER_QUERY_LAUNCH, mrv.MRV_HIERARCHICAL):
        np.testing.assert_array_equal(ctx.mv_validate(ba, flags=fl), v)
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True)
    np.testing.assert_array_equal(v2, v)
    ref = o.mv_min_clearance()
    fin = np.isfinite(ref)
    np.testing.assert_array_equal(np.isfinite(mc), fin)
    np.testing.assert_allclose(mc[fin], ref[fin], atol=PA.CLR_TOL, rtol=0)
    PA.check_mv(o, ctx.mv_validate(ba, flags=mrv.MRV_PRIORITY), priority=True)
    # the same scene without its cylinders is valid at least as often
    bare = copy.deepcopy(w)
    bare.envs[0].cylinders = np.zeros((0, 7), np.float32)
    vb = ctx.mv_validate(ctx.bind(bare))
    assert np.all(vb >= v) and vb.sum() >= v.sum()


def test_discs_past_cylinders(ctx):
    """Discs in the plane z = 0 among vertical cylinders (one lane per state)."""
    rng = np.random.default_rng(43)
    cyl = np.array([[x, y, -1.0, x, y, 1.0, r] for x, y, r in
                    zip(rng.uniform(1, 9, 12), rng.uniform(1, 9, 12), rng.uniform(0.1, 0.6, 12))], np.float32)
    env = W.Env(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), "pillars", cyl)
    bb = W.BatchBuilder(2, True)
    for _ in range(400):
        T = int(rng.integers(5, 150))
        bb.add([0, 0], [np.array([rng.uniform(0, 10, 2), rng.uniform(0, 10, 2)], np.float32) for _ in range(2)],
               [[T]] * 2, 0, 0)
    w = W.Workload("discs_pillars", [W.disc_robot(0.25)], [env], bb.build(0.05), env=0, check_env=True)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    v = ctx.mv_validate(ba)
    n, und = PA.check_mv(o, v)
    assert und < 10 and 0.05 < v.mean() < 0.95
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True)
    np.testing.assert_allclose(mc, o.mv_min_clearance(), atol=PA.CLR_TOL, rtol=0)
    st = ctx.stats()
    assert st["cylinder_tests"] == st["states_checked"] * 2 * len(cyl)


def test_cage8_small(ctx):
    w = W.make_cage8_mv(120)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    PA.check_mv(o, v)
    for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR, mrv.MRV_PAIRS_FIRST,
               mrv.MRV_PAIRS_FIRST | mrv.MRV_NO_BROADPHASE):
        np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=fl)), v)
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True)
    np.testing.assert_array_equal(_np(v2), v)
    np.testing.assert_allclose(_np(mc), o.mv_min_clearance(threads=PA.THREADS), atol=PA.CLR_TOL, rtol=0)
    # dense exhaustive: every test of every state, the cylinder share exact
    ctx.mv_validate(ba, exhaustive=True, flags=mrv.MRV_NO_BROADPHASE)
    st = ctx.stats()
    assert st["sphere_tests"] == st["sphere_tests_available"]
    assert st["cylinder_tests"] == st["states_available"] * 8 * 64 * len(w.envs[0].cylinders)
    per_state = 28 * 64 * 64 + 8 * 1342 + 8 * 64 * len(w.envs[0].cylinders)
    assert st["sphere_tests"] == st["states_available"] * per_state


def test_cage8_full_10k(ctx):
    """The benchmark's size and launch (device batch): all 10,000 motions
    against the oracle."""
    w = W.make_cage8_mv(10000)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    n, _ = PA.check_mv(o, v)
    assert n == 10000


def test_clearance_diagnostic_with_cylinders(ctx):
    w = W.make_cage8_mv(4)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    T = int(o.query_T([1])[0])
    ts = np.array([0, T // 3, T], np.int32)
    got = ctx.clearance(ba, 1, ts, 512)
    ref = o.clearance(1, ts)
    np.testing.assert_allclose(got, ref, atol=PA.CLR_TOL, rtol=0)


def test_cylinder_upload_checks(ctx):
    ok = np.array([[0, 0, 0, 0, 0, 1, 0.1]], np.float32)
    ctx.upload_env(W.Env(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), "ok", ok))
    for bad in ([[0, 0, 0, 0, 0, 0, 0.1]], [[0, 0, 0, 0, 0, 1, -0.1]], [[0, 0, np.nan, 0, 0, 1, 0.1]]):
        with pytest.raises(mrv.MrvError) as e:
            ctx.upload_env(W.Env(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), "bad",
                                 np.array(bad, np.float32)))
        assert "MRV_ERR_ARG" in str(e.value)
