"""Teams beyond 8 robots or 512 spheres (the paper's 16-arm Cage, Sec. V-A)
on the GPU against the oracle.  Such queries run on the large-team kernel
instance; these tests cover random teams of 9-16 robots through every code
path and flag, batches mixing both kernel instances, FFC keys naming pairs
past index 31, a few robots whose sphere count alone exceeds the team
layout, 16 discs (one lane per state), and the floor- and ceiling-mounted
16-arm team in the cylinder cage at small and at full size."""
from __future__ import annotations

import dataclasses

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


@pytest.mark.parametrize("seed", range(3))
def test_random_large_teams(ctx, seed):
    """9-16 random robots per query; every path gives the oracle's answers."""
    w = tiny_workload(1600 + seed, n_queries=40, timed=bool(seed % 2), min_robots=9, max_robots=16,
                      n_models=6, cylinders=3)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    v = ctx.mv_validate(ba)
    PA.check_mv(o, v)
    c = ctx.ffc_find(ba)
    PA.check_ffc(o, c)
    assert (c[:, 2] >= 8).any(), "pair indices beyond one 32-bit mask are exercised"
    for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_PER_QUERY_LAUNCH, mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR,
               mrv.MRV_HIERARCHICAL | mrv.MRV_NO_BROADPHASE, mrv.MRV_PAIRS_FIRST,
               mrv.MRV_PAIRS_FIRST | mrv.MRV_NO_BROADPHASE, mrv.MRV_PAIRS_FIRST | mrv.MRV_PER_QUERY_LAUNCH):
        np.testing.assert_array_equal(ctx.mv_validate(ba, flags=fl), v)
    for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_PER_QUERY_LAUNCH):
        np.testing.assert_array_equal(ctx.ffc_find(ba, flags=fl), c)
    np.testing.assert_array_equal(ctx.ffc_find(ba, exhaustive=True), c)
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True)
    np.testing.assert_array_equal(v2, v)
    ref = o.mv_min_clearance()
    fin = np.isfinite(ref)
    np.testing.assert_array_equal(np.isfinite(mc), fin)
    np.testing.assert_allclose(mc[fin], ref[fin], atol=PA.CLR_TOL, rtol=0)
    PA.check_mv(o, ctx.mv_validate(ba, flags=mrv.MRV_PRIORITY), priority=True)
    # device batch (both instances launched) gives the same answers
    bd = ba.to("cuda")
    np.testing.assert_array_equal(_np(ctx.mv_validate(bd)), v)
    np.testing.assert_array_equal(_np(ctx.ffc_find(bd)), c)


def test_mixed_classes_one_batch(ctx):
    """Queries of 1-16 robots interleaved: both kernel instances in one call,
    each taking only its own work items; the exhaustive statistics count
    every state of both."""
    w = tiny_workload(1700, n_queries=120, timed=True, min_robots=1, max_robots=16, n_models=5, max_steps=12)
    o = O.Oracle(w)
    n_rob = np.diff(w.batch.q_robot_off)
    assert (n_rob > 8).sum() > 20 and (n_rob <= 8).sum() > 20
    ba = ctx.bind(w)
    PA.check_mv(o, ctx.mv_validate(ba))
    PA.check_ffc(o, ctx.ffc_find(ba))
    ctx.mv_validate(ba, exhaustive=True)
    st = ctx.stats()
    assert st["states_checked"] == st["states_available"] == int((o.query_T() + 1).sum())


def test_graph_replay_of_mixed_classes(ctx):
    """A CUDA graph of a batch holding both kernel classes (the large-team
    instance captured on the fork's stream) replays to the direct results."""
    w = tiny_workload(1710, n_queries=150, timed=True, min_robots=1, max_robots=16, n_models=5, max_steps=10)
    ba = ctx.bind(w).to("cuda")
    v1, c1 = ctx.run(ba)
    kind = torch.as_tensor(w.batch.q_kind, device="cuda")
    vg = torch.full_like(v1, 7)
    cg = torch.full_like(c1, 7)
    g = mrv.mrv_graph_create(ctx.h, ba.struct(mrv.MRV_CHECK_ENV, with_kind=True), vg, cg)
    for _ in range(3):
        mrv.mrv_graph_launch(g)
        ctx.sync()
        assert torch.equal(vg[kind == 0], v1[kind == 0])
        assert torch.equal(cg[kind == 1], c1[kind == 1])
    mrv.mrv_graph_destroy(g)
    o = O.Oracle(w)
    PA.check_mv(o, _np(v1)[w.batch.q_kind == 0], np.nonzero(w.batch.q_kind == 0)[0])
    PA.check_ffc(o, _np(c1)[w.batch.q_kind == 1], np.nonzero(w.batch.q_kind == 1)[0])


def test_sphere_count_alone_selects_large_layout(ctx):
    """Three robots of 200 spheres (600 > 512): the large-team instance by
    sphere count, with dense and broadphase paths agreeing with the oracle."""
    rng = np.random.default_rng(1750)
    base = tiny_workload(1750, n_queries=1, n_models=1).models[0]
    reps = 200 // base.n_spheres + 1
    xyzr = np.tile(base.sphere_xyzr, (reps, 1))[:200].copy()
    xyzr[:, :3] += rng.normal(0, 0.01, (200, 3)).astype(np.float32)
    big = dataclasses.replace(base, sphere_xyzr=xyzr, sphere_link=np.tile(base.sphere_link, reps)[:200].copy(),
                              self_pairs=np.zeros((0, 2), np.int32), name="big")
    w0 = tiny_workload(1751, n_queries=30, timed=True, min_robots=3, max_robots=3, n_models=1, max_steps=8)
    w = dataclasses.replace(w0, models=[big])
    o = O.Oracle(w)
    ba = ctx.bind(w)
    v = ctx.mv_validate(ba)
    PA.check_mv(o, v)
    np.testing.assert_array_equal(ctx.mv_validate(ba, flags=mrv.MRV_NO_BROADPHASE), v)
    PA.check_ffc(o, ctx.ffc_find(ba))


def test_sixteen_discs(ctx):
    """16 discs on straight lines across a shared square (one lane per state,
    the large-team instance): FFC conflicts naming late pairs, MV."""
    rng = np.random.default_rng(1760)
    disc = W.disc_robot(0.2)
    bb = W.BatchBuilder(2, True)
    for _ in range(200):
        T = int(rng.integers(20, 120))
        paths = [np.array([rng.uniform(0, 6, 2), rng.uniform(0, 6, 2)], np.float32) for _ in range(16)]
        bb.add([0] * 16, paths, [[T]] * 16, int(rng.integers(0, 2)), -1)
    w = W.Workload("discs16", [disc], [], bb.build(0.05), env=-1, check_env=False)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    c = ctx.ffc_find(ba)
    PA.check_ffc(o, c)
    assert c[:, 1].max() >= 8
    PA.check_mv(o, ctx.mv_validate(ba, check_env=False))
    v, c2 = ctx.run(ba)
    kind = w.batch.q_kind
    np.testing.assert_array_equal(_np(c2)[kind == 1], _np(ctx.ffc_find(ba))[kind == 1])


def test_cage16_small(ctx):
    w = W.make_cage16_mv(100)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    PA.check_mv(o, v)
    assert 0 < v.sum() < len(v)
    for fl in (mrv.MRV_NO_BROADPHASE, mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR, mrv.MRV_PER_QUERY_LAUNCH,
               mrv.MRV_PAIRS_FIRST, mrv.MRV_PAIRS_FIRST | mrv.MRV_NO_BROADPHASE):
        np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=fl)), v)
        st = ctx.stats()
        assert 0 < st["states_checked"] <= st["states_available"]
    v2, mc = ctx.mv_validate(ba, exhaustive=True, min_clearance=True)
    np.testing.assert_array_equal(_np(v2), v)
    np.testing.assert_allclose(_np(mc), o.mv_min_clearance(threads=PA.THREADS), atol=PA.CLR_TOL, rtol=0)
    # dense exhaustive: every test of every state (120 pairs of 64 x 64 spheres)
    ctx.mv_validate(ba, exhaustive=True, flags=mrv.MRV_NO_BROADPHASE)
    st = ctx.stats()
    n_cyl = len(w.envs[0].cylinders)
    per_state = 120 * 64 * 64 + 16 * 1342 + 16 * 64 * n_cyl
    assert st["sphere_tests"] == st["sphere_tests_available"] == st["states_available"] * per_state
    wf = W.make_cage16_ffc(100)
    of = O.Oracle(wf)
    cf = _np(ctx.ffc_find(ctx.bind(wf).to("cuda")))
    PA.check_ffc(of, cf)


def test_cage16_full_10k(ctx):
    """The benchmark's sizes and launches (device batches): all 10,000 MV
    edges and 2,000 of the 10,000 FFC motions (a seeded sample; each costs
    the oracle about 120 robot pairs x 4,096 sphere pairs per state) against
    the oracle."""
    w = W.make_cage16_mv(10000)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    n, _ = PA.check_mv(o, v)
    assert n == 10000
    wf = W.make_cage16_ffc(10000)
    of = O.Oracle(wf)
    c = _np(ctx.ffc_find(ctx.bind(wf).to("cuda")))
    n, _ = PA.check_ffc(of, c, idx=PA.sample(wf.batch.n_queries, 2000, seed=10))
    assert n == 2000


def test_clearance_diagnostic_sixteen_arms(ctx):
    w = W.make_cage16_mv(3, edge=None)
    o = O.Oracle(w)
    ba = ctx.bind(w)
    T = int(o.query_T([2])[0])
    ts = np.array([0, T // 2, T], np.int32)
    got = ctx.clearance(ba, 2, ts, 1024)
    np.testing.assert_allclose(got, o.clearance(2, ts), atol=PA.CLR_TOL, rtol=0)


def test_server_mixes_team_and_large_requests():
    """16-arm and 8-arm requests through the continuous-batching server from
    several client threads (micro-batches holding both kernel classes, the
    large-team instance on each stream's fork): the results of every request
    equal those of running it alone."""
    import threading
    c = mrv.Context(0)
    reqs = []
    for w in (W.make_cage16_mv(400), W.make_cage8_mv(400)):
        rids = [c.upload_model(m) for m in w.models]
        eids = [c.upload_env(e) for e in w.envs]
        ba = c.bind(w, rids, eids)
        reqs += [mrv.slice_batch(ba, q0, q0 + 50) for q0 in range(0, 400, 50)]
    alone = [c.run(r) for r in reqs]
    srv = mrv.Server(c, n_streams=3, device_budget_bytes=256 << 20, max_batch_queries=200, max_pending=100)
    got = [None] * len(reqs)

    def client(ids):
        for i in ids:
            t = srv.submit(reqs[i])
            got[i] = srv.wait(t, reqs[i].n_queries, timeout_ms=60000)

    th = [threading.Thread(target=client, args=(list(range(k, len(reqs), 4)),)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st = srv.stats()
    srv.close()
    for (va, _), (vm, _) in zip(alone, got):
        np.testing.assert_array_equal(_np(va), _np(vm))
    assert st["completed"] == len(reqs)
    c.close()


@pytest.mark.parametrize("n_arms", [4, 8, 16])
@pytest.mark.parametrize("obstacles", [True, False])
def test_validation_study_motions(ctx, n_arms, obstacles):
    """The validation study's motions (4, 8 and 16 arms between whole-team
    valid configurations, with and without obstacles): every order against
    the oracle, early-terminating and exhaustive."""
    w = W.make_cage_team_study(n_arms, 120, obstacles=obstacles)
    o = O.Oracle(w)
    ba = ctx.bind(w).to("cuda")
    v = _np(ctx.mv_validate(ba))
    PA.check_mv(o, v)
    for fl in (mrv.MRV_HIERARCHICAL, mrv.MRV_LINEAR, mrv.MRV_HIERARCHICAL | mrv.MRV_LINEAR, mrv.MRV_NO_BROADPHASE):
        np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=fl)), v)
        np.testing.assert_array_equal(_np(ctx.mv_validate(ba, flags=fl, exhaustive=True)), v)
        st = ctx.stats()
        assert st["states_checked"] == st["states_available"]
