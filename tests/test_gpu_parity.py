"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small cases are compared query by query in full (several 32-state tiles,
ragged path lengths, every robot kind); the full-size workloads run in the
launch configuration the benchmark times and are checked on sampled queries
the oracle computes one by one.  Exact match is required on MV booleans and
FFC (t, i, j) for every query whose oracle clearances keep 1e-4 m from zero;
clearance values must agree within 1e-5 m.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_23960_gb300 import mrv
from paper_2604_23960_gb300 import workloads as W
from tests import parity as PA
from tests.tiny import tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = mrv.Context(0)
    yield c
    c.close()


def _np(x):
    return x if isinstance(x, np.ndarray) else x.cpu().numpy()


# ------------------------------------------------------------------ tiny cases

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("timed", [True, False])
def test_tiny_mv_ffc(ctx, seed, timed):
    w = tiny_workload(1000 + seed, n_queries=40, timed=timed, max_steps=40, max_robots=4)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    for ce in (True, False):
        v = ctx.mv_validate(ba, check_env=ce)
        PA.check_mv(o, v, check_env=ce)
        ve = ctx.mv_validate(ba, check_env=ce, exhaustive=True)
        np.testing.assert_array_equal(v, ve)
    c = ctx.ffc_find(ba)
    PA.check_ffc(o, c)
    np.testing.assert_array_equal(ctx.ffc_find(ba, exhaustive=True), c)
    # device-resident batch: identical results
    bd = ba.to("cuda")
    np.testing.assert_array_equal(_np(ctx.mv_validate(bd)), ctx.mv_validate(ba))
    np.testing.assert_array_equal(_np(ctx.ffc_find(bd)), c)
    # hierarchical order (Alg. 1), the linear state map and the pairs-first
    # order (adjacent fixed-base pairs first): same verdicts
    for fl in (mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR, mrv.MRV_LINEAR | mrv.MRV_HIERARCHICAL, mrv.MRV_PAIRS_FIRST,
               mrv.MRV_PAIRS_FIRST | mrv.MRV_LINEAR, mrv.MRV_PAIRS_FIRST | mrv.MRV_NO_BROADPHASE):
        for ce in (True, False):
            np.testing.assert_array_equal(ctx.mv_validate(ba, check_env=ce, flags=fl),
                                          ctx.mv_validate(ba, check_env=ce))
    np.testing.assert_array_equal(ctx.ffc_find(ba, flags=mrv.MRV_LINEAR), c)   # FFC is linear already
    # every sphere pair tested (no frame-level broadphase): same verdicts
    for ce in (True, False):
        np.testing.assert_array_equal(ctx.mv_validate(ba, check_env=ce, flags=mrv.MRV_NO_BROADPHASE),
                                      ctx.mv_validate(ba, check_env=ce))
    np.testing.assert_array_equal(ctx.ffc_find(ba, flags=mrv.MRV_NO_BROADPHASE), c)
    # one synchronous launch per query: identical results
    np.testing.assert_array_equal(ctx.mv_validate(ba, flags=mrv.MRV_PER_QUERY_LAUNCH), ctx.mv_validate(ba))
    np.testing.assert_array_equal(ctx.ffc_find(ba, flags=mrv.MRV_PER_QUERY_LAUNCH), c)


@pytest.mark.parametrize("seed", range(4))
def test_tiny_min_clearance(ctx, seed):
    w = tiny_workload(1100 + seed, n_queries=30, timed=True, max_steps=30)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    for ce in (True, False):
        v, mc = ctx.mv_validate(ba, check_env=ce, exhaustive=True, min_clearance=True)
        ref = o.mv_min_clearance(check_env=ce)
        fin = np.isfinite(ref)
        np.testing.assert_array_equal(np.isfinite(mc), fin)
        np.testing.assert_allclose(mc[fin], ref[fin], atol=PA.CLR_TOL, rtol=0)


def test_many_robots_mixed_kinds(ctx):
    """Up to 8 robots per query, DH chains mixed with point robots."""
    w = tiny_workload(1200, n_queries=60, timed=True, max_robots=8, n_models=8, max_steps=20)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    PA.check_mv(o, ctx.mv_validate(ba))
    PA.check_ffc(o, ctx.ffc_find(ba))


def test_clearance_diagnostic(ctx):
    w = tiny_workload(1300, n_queries=8, timed=True, max_steps=12)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    T = o.query_T()
    for q in range(w.batch.n_queries):
        ts = list(range(0, int(T[q]) + 1, max(1, int(T[q]) // 5)))
        M = sum(w.models[w.batch.slot_robot[s]].n_spheres
                for s in range(w.batch.q_robot_off[q], w.batch.q_robot_off[q + 1]))
        for ce in (True, False):
            got = ctx.clearance(ba, q, ts, M, check_env=ce)
            ref = o.clearance(q, ts, check_env=ce)
            fin = np.isfinite(ref)
            np.testing.assert_array_equal(np.isfinite(got), fin)
            np.testing.assert_allclose(got[fin], ref[fin], atol=PA.CLR_TOL, rtol=0)


# ------------------------------------------------- workload-shaped small cases

def test_discs_full(ctx):
    """Two disc robots in the box world: all 1,000 queries, MV and FFC."""
    w = W.make_plain_discs(1000)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    c = _np(ctx.ffc_find(ba))
    _, und_mv = PA.check_mv(o, v)
    _, und_ffc = PA.check_ffc(o, c)
    assert und_mv < 5 and und_ffc < 5
    st = ctx.stats()
    assert st["states_checked"] <= st["states_available"]


def test_cage_mv_small_exhaustive(ctx):
    w = W.make_cage_mv(96)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    PA.check_mv(o, v)
    np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=mrv.MRV_HIERARCHICAL)), v)
    np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=mrv.MRV_NO_BROADPHASE)), v)
    # the four visiting orders (combined / hierarchical x rake / linear): same
    # verdicts; early exit checks a subset of the states, exhaustive all
    for fl in (0, mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR, mrv.MRV_HIERARCHICAL | mrv.MRV_LINEAR,
               mrv.MRV_PAIRS_FIRST, mrv.MRV_PAIRS_FIRST | mrv.MRV_LINEAR):
        for bp in (0, mrv.MRV_NO_BROADPHASE):
            np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=fl | bp)), v)
            st = ctx.stats()
            assert 0 < st["states_checked"] <= st["states_available"]
            np.testing.assert_array_equal(_np(ctx.mv_validate(ba, exhaustive=True, flags=fl | bp)), v)
            st = ctx.stats()
            assert st["states_checked"] == st["states_available"]
            if bp:
                assert st["sphere_tests"] == st["sphere_tests_available"]
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True)
    np.testing.assert_array_equal(_np(v2), v)
    ref = o.mv_min_clearance(threads=PA.THREADS)
    np.testing.assert_allclose(_np(mc), ref, atol=PA.CLR_TOL, rtol=0)
    st = ctx.stats()
    assert st["states_checked"] == st["states_available"]
    ctx.mv_validate(ba, exhaustive=True, flags=mrv.MRV_NO_BROADPHASE)
    st = ctx.stats()
    assert st["sphere_tests"] == st["sphere_tests_available"]


def test_cage_ffc_small(ctx):
    w = W.make_cage_ffc(64)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    c = _np(ctx.ffc_find(ba))
    PA.check_ffc(o, c)
    np.testing.assert_array_equal(_np(ctx.ffc_find(ba, flags=mrv.MRV_NO_BROADPHASE)), c)
    np.testing.assert_array_equal(_np(ctx.ffc_find(ba, exhaustive=True)), c)


def test_ragged_teams_small_mixed(ctx):
    w = W.make_ragged_teams(400, seed=905)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v, c = ctx.run(ba)
    v, c = _np(v), _np(c)
    kind = w.batch.q_kind
    mv_idx, ffc_idx = np.nonzero(kind == 0)[0], np.nonzero(kind == 1)[0]
    PA.check_mv(o, v[mv_idx], mv_idx)
    PA.check_ffc(o, c[ffc_idx], ffc_idx)
    # the same queries through the single-kind entry points
    np.testing.assert_array_equal(_np(ctx.mv_validate(ba))[mv_idx], v[mv_idx])
    np.testing.assert_array_equal(_np(ctx.ffc_find(ba))[ffc_idx], c[ffc_idx])


# --------------------------------------------------------------- edge cases

def _one_query(models, paths, steps=None, env=None, res=0.1, check_env=True):
    bb = W.BatchBuilder(max(m.dof for m in models), steps is not None)
    bb.add(list(range(len(models))), paths, steps, 0, 0 if env is not None else -1)
    return W.Workload("edge", models, [env] if env is not None else [], bb.build(res), 0 if env is not None else -1,
                      check_env)


def test_empty_batch(ctx):
    w = W.make_plain_discs(4)
    ba = ctx.bind(w)
    ba.n_queries = 0
    assert ctx.mv_validate(ba).shape == (0,)
    assert ctx.ffc_find(ba).shape == (0, 3)


def test_single_robot_and_stationary(ctx):
    env = W.world_boxes(3)
    d = W.disc_robot(0.25)
    # one robot: FFC has no pair, MV checks obstacles only
    w = _one_query([d], [np.array([[0.1, 0.1], [9.9, 9.9]])], env=env)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    PA.check_mv(o, ctx.mv_validate(ba))
    assert list(ctx.ffc_find(ba)[0]) == [-1, -1, -1]
    # no motion at all: T = 0, one state
    w0 = _one_query([d, d], [np.array([[1.0, 1.0], [1.0, 1.0]]), np.array([[1.2, 1.0], [1.2, 1.0]])])
    assert O.Oracle(w0).query_T()[0] == 0
    ba0 = ctx.bind(w0)
    assert ctx.mv_validate(ba0)[0] == 0
    assert list(ctx.ffc_find(ba0)[0]) == [0, 0, 1]


def test_eight_arms_max_spheres(ctx):
    """8 arms x 64 spheres = 512 spheres, the per-query maximum."""
    fx = W.load_cage_fixtures()
    arms = [W.panda_like(W._pose(1.3 * np.cos(a), 1.3 * np.sin(a), 0.0, a + np.pi), fx["self_pairs"])
            for a in np.linspace(0, 2 * np.pi, 8, endpoint=False)]
    rng = np.random.default_rng(5)
    bb = W.BatchBuilder(7, True)
    for _ in range(6):
        paths = [rng.uniform(W.PANDA_LO, W.PANDA_HI, (3, 7)) for _ in arms]
        bb.add(list(range(8)), paths, [rng.integers(10, 40, 2) for _ in arms], 0, -1)
    w = W.Workload("eight", arms, [], bb.build(), -1, True)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    PA.check_mv(o, ctx.mv_validate(ba))
    PA.check_ffc(o, ctx.ffc_find(ba))


def test_errors_are_reported(ctx):
    w = W.make_plain_discs(4)
    ba = ctx.bind(w)
    bad = ba.a["slot_robot_id"].copy()
    bad[1] = 12345
    ba2 = mrv.BatchArrays(dict(ba.a, slot_robot_id=bad), ba.n_queries, ba.n_slots, ba.n_waypoints, ba.wp_stride,
                          ba.resolution, ba.env_id, False)
    with pytest.raises(mrv.MrvError) as e:
        ctx.mv_validate(ba2)
    assert e.value.code == -3
    # timed form needs >= 1 step per segment
    wt = tiny_workload(7, n_queries=3, timed=True)
    bt = ctx.bind(wt)
    st = bt.a["seg_steps"].copy()
    st[0] = 0
    bt2 = mrv.BatchArrays(dict(bt.a, seg_steps=st), bt.n_queries, bt.n_slots, bt.n_waypoints, bt.wp_stride,
                          bt.resolution, bt.env_id, False)
    if wt.batch.slot_wp_off[1] - wt.batch.slot_wp_off[0] > 1:
        with pytest.raises(mrv.MrvError):
            ctx.ffc_find(bt2)
    # too many robots in a query
    d = W.disc_robot(0.1)
    n = mrv.MRV_MAX_ROBOTS + 1
    over = _one_query([d] * n, [np.array([[i, 0.0], [i, 1.0]]) for i in range(n)])
    with pytest.raises(mrv.MrvError) as e:
        ctx.mv_validate(ctx.bind(over))
    assert e.value.code == -7
    # too many spheres in a query (five 256-sphere robots), host and device batch
    d1 = W.disc_robot(0.05)
    big = dataclasses.replace(d1, sphere_xyzr=np.tile(d1.sphere_xyzr, (256, 1)),
                              sphere_link=np.tile(d1.sphere_link, 256), name="big")
    five = _one_query([big] * 5, [np.array([[i, 0.0], [i, 1.0]]) for i in range(5)])
    for dev in (False, True):
        b5 = ctx.bind(five)
        with pytest.raises(mrv.MrvError) as e:
            ctx.mv_validate(b5.to("cuda") if dev else b5)
        assert e.value.code == -7
    # the pairs-first order excludes the hierarchical order and the prioritized MV
    for fl in (mrv.MRV_PAIRS_FIRST | mrv.MRV_HIERARCHICAL, mrv.MRV_PAIRS_FIRST | mrv.MRV_PRIORITY):
        with pytest.raises(mrv.MrvError) as e:
            ctx.mv_validate(ba, flags=fl)
        assert e.value.code == -1
    # the context stays usable
    PA.check_mv(O.Oracle(w), ctx.mv_validate(ba))


def test_repeatable_and_graph_replay(ctx):
    import torch
    w = W.make_ragged_teams(3000, seed=77)
    ba = ctx.bind(w).to("cuda")
    kind = torch.as_tensor(w.batch.q_kind, device="cuda")
    v1, c1 = ctx.run(ba)
    v2, c2 = ctx.run(ba)
    # mrv_run writes valid_out for MV queries and conflict_out for FFC queries
    assert torch.equal(v1[kind == 0], v2[kind == 0]) and torch.equal(c1[kind == 1], c2[kind == 1])
    vg = torch.full_like(v1, 7)
    cg = torch.full_like(c1, 7)
    g = mrv.mrv_graph_create(ctx.h, ba.struct(mrv.MRV_CHECK_ENV, with_kind=True), vg, cg)
    for _ in range(3):
        mrv.mrv_graph_launch(g)
        ctx.sync()
        assert torch.equal(vg[kind == 0], v1[kind == 0])
        assert torch.equal(cg[kind == 1], c1[kind == 1])
    mrv.mrv_graph_destroy(g)


def test_tunings_do_not_change_results(ctx, tmp_path):
    import torch
    w = W.make_ragged_teams(2000, seed=78)
    ba = ctx.bind(w).to("cuda")
    mvq = torch.as_tensor(w.batch.q_kind == 0, device="cuda")
    ffq = ~mvq

    def same(a, b):   # mrv_run leaves the other kind's output untouched
        return torch.equal(a[0][mvq], b[0][mvq]) and torch.equal(a[1][ffq], b[1][ffq])

    ref = ctx.run(ba)
    saved = mrv.mrv_get_tuning(ctx.h)
    try:
        for ch, wp, sp, mo in [(1, 2, 1, 0), (2, 8, 2, 1), (16, 4, 8, 0), (3, 12, 4, 1), (1, 1, 4, 0),
                               (1, 4, 16, 1), (2, 6, 32, 0)]:
            mrv.mrv_set_tuning(ctx.h, ch, wp, 0, sp, mo)
            assert same(ctx.run(ba), ref)
        # the tuned MV order (1: hierarchical) is the order of early-exit
        # batches naming none; exhaustive runs keep the combined order (fewer
        # work items: one phase per slice) unless the flag names it
        mrv.mrv_set_tuning(ctx.h, 1, 4, 0, 4, 1)
        ctx.run(ba, exhaustive=True)
        items_tuned_ex = ctx.stats()["work_items"]
        ctx.run(ba, exhaustive=True, flags=mrv.MRV_HIERARCHICAL)
        items_hier_ex = ctx.stats()["work_items"]
        mrv.mrv_set_tuning(ctx.h, 1, 4, 0, 4, 0)
        ctx.run(ba, exhaustive=True)
        assert ctx.stats()["work_items"] == items_tuned_ex < items_hier_ex
        # early exit with the tuned order runs two phases: the MV queries'
        # verdicts are those of the combined order
        mrv.mrv_set_tuning(ctx.h, 1, 4, 0, 4, 1)
        assert same(ctx.run(ba), ref)
        with pytest.raises(mrv.MrvError):
            mrv.mrv_set_tuning(ctx.h, 1, 4, 0, 4, 2)
        t = mrv.mrv_autotune(ctx.h, ba.struct(mrv.MRV_CHECK_ENV, with_kind=True), str(tmp_path / "tune.txt"))
        assert t["slices_per_item"] >= 1 and t["warps_per_block"] >= 1
        assert (tmp_path / "tune.txt").read_text().strip()
        t2 = mrv.mrv_autotune(ctx.h, ba.struct(mrv.MRV_CHECK_ENV, with_kind=True), str(tmp_path / "tune.txt"))
        assert t2 == t   # cached
        assert same(ctx.run(ba), ref)
    finally:
        mrv.mrv_set_tuning(ctx.h, saved["slices_per_item"], saved["warps_per_block"], saved["blocks_per_sm"],
                           saved["tile_split"], saved["mv_order"])


# --------------------------------------------- full sizes, benchmark launches

def test_full_cage_mv_10k(ctx):
    """Every one of the 10,000 cage motions against the oracle."""
    w = W.make_cage_mv(10000)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    n, _ = PA.check_mv(O.Oracle(w), v)
    assert n == 10000


def test_full_cage_ffc_100k(ctx):
    """100k path-sets in one launch; 10,000 of them (a seeded sample) against
    the oracle, the rest checked for well-formed answers."""
    w = W.make_cage_ffc(100000)
    ba = ctx.bind(w).to("cuda")
    c = _np(ctx.ffc_find(ba))
    idx = PA.sample(w.batch.n_queries, 10000, seed=2)
    n, _ = PA.check_ffc(O.Oracle(w), c[idx], idx)
    assert n == 10000
    # every reported conflict time lies inside its query
    T = c[:, 0]
    assert np.all((T == -1) | (T >= 0))
    assert np.all((c[:, 1] < c[:, 2]) | (c[:, 0] == -1))


def test_full_ragged_1m(ctx):
    w = W.make_ragged_teams(1_000_000)
    ba = ctx.bind(w).to("cuda")
    v, c = ctx.run(ba)
    v, c = _np(v), _np(c)
    idx = PA.sample(w.batch.n_queries, 50000, seed=3)
    kind = w.batch.q_kind[idx]
    o = O.Oracle(w)
    n_mv, _ = PA.check_mv(o, v[idx[kind == 0]], idx[kind == 0])
    n_ffc, _ = PA.check_ffc(o, c[idx[kind == 1]], idx[kind == 1])
    assert n_mv + n_ffc == 50000


def test_longest_motions(ctx):
    """T = MRV_MAX_STEPS (2^24 states, t = 0..2^24 - 1): disc 0 drifts slowly far from a
    stationary disc 1, then jumps onto it in a one-step segment, so the only
    conflict is the last state (decidable); a second query jumps to a clear
    spot instead (valid, compared on its exhaustive minimum clearance); one
    step more than the limit is rejected."""
    T = mrv.MRV_MAX_STEPS
    assert T == (1 << 24) - 1
    disc = W.disc_robot(0.25)
    bb = W.BatchBuilder(2, True)
    for end in ((5.0, 5.0), (3.0, 3.0)):
        bb.add([0, 0], [np.array([(1.0, 1.0), (1.0, 2.0), end], np.float32),
                        np.array([(5.0, 5.0), (5.0, 5.0)], np.float32)], [[T - 1, 1], [T]])
    w = W.Workload("long", [disc], [], bb.build(0.05), env=-1, check_env=False)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    assert list(o.query_T()) == [T, T]
    c = ctx.ffc_find(ba)
    np.testing.assert_array_equal(c, o.ffc(threads=2))
    assert tuple(c[0]) == (T, 0, 1) and tuple(c[1]) == (-1, -1, -1)
    v = ctx.mv_validate(ba, check_env=False)
    assert list(v) == [0, 1]
    v2, mc = ctx.mv_validate(ba, check_env=False, exhaustive=True, min_clearance=True)
    np.testing.assert_allclose(mc, o.mv_min_clearance(check_env=False, threads=2), atol=PA.CLR_TOL, rtol=0)
    st = ctx.stats()
    assert st["states_checked"] == st["states_available"] == 2 * (T + 1)
    bb = W.BatchBuilder(2, True)
    bb.add([0, 0], [np.array([(1.0, 1.0), (2.0, 2.0)], np.float32), np.array([(5.0, 5.0), (5.0, 5.0)], np.float32)],
           [[T + 1], [1]])
    with pytest.raises(mrv.MrvError):
        ctx.ffc_find(ctx.bind(W.Workload("toolong", [disc], [], bb.build(0.05), env=-1, check_env=False)))


def test_ffc_repeatable_under_concurrent_claims(ctx):
    """FFC work items of one query run on many warps at once, and a warp may
    check an item's liveness long after claiming it; an item may only be
    skipped for a conflict before its own first state.  Repeated runs of
    long timed paths (and of both MV orders on mixed batches) give identical
    first conflicts, equal to the oracle's on a sample."""
    w = W.make_cage_ffc(20000, query_seed=41)
    ba = ctx.bind(w).to("cuda")
    ref = _np(ctx.ffc_find(ba))
    for _ in range(6):
        np.testing.assert_array_equal(_np(ctx.ffc_find(ba)), ref)
    idx = PA.sample(w.batch.n_queries, 2000, seed=3)
    PA.check_ffc(O.Oracle(w), ref[idx], idx)
    wr = W.make_ragged_teams(20000, seed=79)
    br = ctx.bind(wr).to("cuda")
    kind = wr.batch.q_kind
    v0, c0 = (_np(x) for x in ctx.run(br))
    for fl in (0, mrv.MRV_HIERARCHICAL, 0, mrv.MRV_HIERARCHICAL):
        v, c = (_np(x) for x in ctx.run(br, flags=fl))
        np.testing.assert_array_equal(v[kind == 0], v0[kind == 0])
        np.testing.assert_array_equal(c[kind == 1], c0[kind == 1])


@pytest.mark.parametrize("gridless", [False, True])
def test_obstacle_lists_without_a_grid_cell(gridless):
    """Frames that no grid cell covers scan every obstacle of the
    environment: frames larger than the grid's radius (the environment is
    uploaded before the models, so its grid is built for 0.3 m frames and the
    discs' frames are 0.45 and 0.6 m), and an environment with more obstacle
    spheres than a grid indexes (70,000, most of them above the discs' plane:
    no grid at all).  MV verdicts (a mix of valid and colliding motions) and
    FFC conflicts equal the oracle's, with and without the frame broadphase."""
    rng = np.random.default_rng(1400 + int(gridless))
    env = W.world_boxes(7, n=8)
    if gridless:
        n = 70000   # above the 65,535 obstacles of one kind a grid indexes
        z = np.where(np.arange(n) < 10, 0.0, rng.uniform(0.7, 3.0, n))
        sph = np.column_stack([rng.uniform(0.0, 10.0, n), rng.uniform(0.0, 10.0, n), z,
                               np.full(n, 0.03)]).astype(np.float32)
        env = W.Env(sph, env.aabbs, name="many")
    discs = [W.disc_robot(0.6), W.disc_robot(0.45)]
    bb = W.BatchBuilder(2, False)
    for _ in range(60):
        robots = [int(rng.integers(0, 2)) for _ in range(int(rng.integers(1, 4)))]
        paths = []
        for _r in robots:
            a = rng.uniform(0.5, 9.5, 2)
            paths.append(np.array([a, np.clip(a + rng.uniform(-1.0, 1.0, 2), 0.5, 9.5)]))
        bb.add(robots, paths, None, int(rng.integers(0, 2)), 0)
    w = W.Workload("beyond_grid", discs, [env], bb.build(0.1), env=0, check_env=True)
    c = mrv.Context(0)
    try:
        eid = c.upload_env(env)
        rids = [c.upload_model(m) for m in discs]
        ba = c.bind(w, rids, [eid])
        o = O.Oracle(w)
        v = c.mv_validate(ba)
        PA.check_mv(o, v, check_env=True)
        assert 0 < int(np.sum(v)) < len(v)
        np.testing.assert_array_equal(c.mv_validate(ba, flags=mrv.MRV_NO_BROADPHASE), v)
        f = c.ffc_find(ba)
        PA.check_ffc(o, f)
        np.testing.assert_array_equal(c.ffc_find(ba, flags=mrv.MRV_NO_BROADPHASE), f)
    finally:
        c.close()


def test_overflowing_candidate_lists_go_to_the_full_instance(ctx):
    """States whose broadphase candidate lists overflow (more than 64
    frame-obstacle or frame-frame candidates at one state) are handed from
    the default kernel instance to the full one, which reruns every item of
    the query with its in-lane fallbacks: a Panda-like arm inside a dense
    cloud of obstacle spheres (MV), and three arms on one base with five
    discs around it (FFC and MV).  Results equal the oracle's and the
    broadphase-free run's, and the statistics count the queries handed over.
    Eight arms on a 1 m circle (the team class, which keeps the in-lane
    fallbacks) give the oracle's conflicts too."""
    fx = W.load_cage_fixtures()
    rng = np.random.default_rng(1500)
    arm = W.panda_like(W._pose(0.0, 0.0, 0.0), fx["self_pairs"])
    n = 1500
    cloud = np.column_stack([rng.uniform(-0.9, 0.9, n), rng.uniform(-0.9, 0.9, n), rng.uniform(0.0, 1.3, n),
                             np.full(n, 0.02)]).astype(np.float32)
    env = W.Env(cloud, np.zeros((0, 6), np.float32), name="cloud")
    bb = W.BatchBuilder(7, False)
    for _ in range(24):
        bb.add([0], [rng.uniform(W.PANDA_LO, W.PANDA_HI, (2, 7))], None, 0, 0)
    w = W.Workload("cloud", [arm], [env], bb.build(1.0 / 16), env=0, check_env=True)
    ba = ctx.bind(w)
    v = ctx.mv_validate(ba)
    assert ctx.stats()["queries_redone"] > 0
    PA.check_mv(O.Oracle(w), v, check_env=True)
    np.testing.assert_array_equal(ctx.mv_validate(ba, flags=mrv.MRV_NO_BROADPHASE), v)
    # three arms on one base and five discs around it (197 spheres: the
    # small-team class): far more than 64 overlapping frame pairs per state
    team = [W.panda_like(W._pose(0.0, 0.0, 0.0, yaw), fx["self_pairs"]) for yaw in (0.0, 2.1, 4.2)]
    team += [W.disc_robot(0.3, z0=0.5, lo=(-0.2, -0.2), hi=(0.2, 0.2)) for _ in range(5)]
    bb = W.BatchBuilder(7, True)
    for _ in range(12):
        paths = [rng.uniform(W.PANDA_LO, W.PANDA_HI, (3, 7)) for _ in range(3)]
        paths += [rng.uniform(-0.2, 0.2, (3, 2)) for _ in range(5)]
        bb.add(list(range(8)), paths, [rng.integers(10, 40, 2) for _ in range(8)], 1, -1)
    w8 = W.Workload("packed_team", team, [], bb.build(), -1, True)
    o8 = O.Oracle(w8)
    b8 = ctx.bind(w8)
    c = ctx.ffc_find(b8)
    assert ctx.stats()["queries_redone"] > 0
    PA.check_ffc(o8, c)
    np.testing.assert_array_equal(ctx.ffc_find(b8, flags=mrv.MRV_NO_BROADPHASE), c)
    v8 = ctx.mv_validate(b8, check_env=False)
    PA.check_mv(o8, v8, check_env=False)
    np.testing.assert_array_equal(ctx.mv_validate(b8, check_env=False, flags=mrv.MRV_NO_BROADPHASE), v8)
    # a looser circle (1 m): conflicts at varied times, lists that may or
    # may not overflow; the same results either way
    rng = np.random.default_rng(1501)
    arms = [W.panda_like(W._pose(np.cos(a), np.sin(a), 0.0, a + np.pi), fx["self_pairs"])
            for a in np.linspace(0, 2 * np.pi, 8, endpoint=False)]
    bb = W.BatchBuilder(7, True)
    for _ in range(12):
        paths = [rng.uniform(W.PANDA_LO, W.PANDA_HI, (3, 7)) for _ in arms]
        bb.add(list(range(8)), paths, [rng.integers(10, 40, 2) for _ in arms], 1, -1)
    w1 = W.Workload("eight_1m", arms, [], bb.build(), -1, True)
    b1 = ctx.bind(w1)
    c1 = ctx.ffc_find(b1)
    PA.check_ffc(O.Oracle(w1), c1)
    np.testing.assert_array_equal(ctx.ffc_find(b1, flags=mrv.MRV_NO_BROADPHASE), c1)
