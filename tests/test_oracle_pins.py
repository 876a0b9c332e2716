"""Pins of the FP64 oracle against facts fixed outside it.

* FK: closed forms of one- and two-joint chains, the modified-DH origin
  formula, base transforms of point robots, the Panda zero pose (public
  kinematics, tests/golden/panda_zero_pose.json).
* CC: sphere-box distance inside / on a face / edge / corner; 3-4-5 spheres.
* Discretisation: step counts from the resolution (Sec. IV-A3) in closed form.
* MV / FFC: brute force on tiny inputs through the paper's own orders
  (Alg. 1 combined and hierarchical, rake and linear, W in {1,4,8,32};
  Alg. 2 with W in {1,4,8,32}), exhaustive conflict enumeration, the
  closed-form first conflict of linearly moving discs, the hand-worked
  head-on example (tests/golden/head_on_discs.json), the rake lane map of
  Fig. 2 (tests/golden/fig2_rake_example.json), and invariants: robot
  permutation, motion reversal, padding = holding the last configuration,
  obstacles do not change FFC, MV without environment is false exactly when
  FFC finds a conflict.
* The first conflict deeper than a bound (what an undecidable FFC answer
  must not pass over): exhaustive enumeration below the bound, the
  closed-form discs with the contact distance moved by the bound, and FFC of
  the same robots with every radius shrunk by half the margin.
"""
from __future__ import annotations

import copy
import json
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_23960_gb300 import workloads as W
from tests import bruteforce as BF
from tests.tiny import tiny_workload

GOLD = Path(__file__).resolve().parent / "golden"


def _one_joint(a, alpha, d, theta0, local):
    m = W.RobotModel(W.KIND_DH, 1, np.array([[a, alpha, d, theta0]], np.float32), None,
                     np.array([-4.0], np.float32), np.array([4.0], np.float32), W._identity34(), 0.0,
                     np.array([1], np.int32), np.array([[*local, 0.1]], np.float32), np.zeros((0, 2), np.int32))
    return m


# --------------------------------------------------------------------------- FK

@pytest.mark.parametrize("q", [0.0, 0.3, -1.2, 2.9])
def test_fk_single_revolute_circle(q):
    L = 0.7
    m = _one_joint(0.0, 0.0, 0.0, 0.0, (L, 0.0, 0.0))
    c = O.fk(m, [q])[0]
    np.testing.assert_allclose(c, [L * math.cos(q), L * math.sin(q), 0.0], atol=1e-7)


@pytest.mark.parametrize("alpha", [0.0, math.pi / 2, -math.pi / 2, 0.7])
def test_fk_general_joint_closed_form(alpha):
    a, d, th0, L, q = 0.1, 0.2, 0.25, 0.3, 0.4
    m = _one_joint(a, alpha, d, th0, (L, 0.0, 0.0))
    a, alpha, d, th0 = (float(np.float32(v)) for v in (a, alpha, d, th0))
    L = float(np.float32(L))
    th = th0 + q
    # origin of the joint frame: (a, -sin(alpha) d, cos(alpha) d); its x axis:
    # (cos th, sin th cos alpha, sin th sin alpha)
    expect = [a + L * math.cos(th),
              -math.sin(alpha) * d + L * math.sin(th) * math.cos(alpha),
              math.cos(alpha) * d + L * math.sin(th) * math.sin(alpha)]
    np.testing.assert_allclose(O.fk(m, [q])[0], expect, atol=1e-7)


def test_fk_two_link_planar():
    L1, L2 = 0.5, 0.3
    m = W.RobotModel(W.KIND_DH, 2, np.array([[0, 0, 0, 0], [L1, 0, 0, 0]], np.float32), None,
                     np.array([-4, -4], np.float32), np.array([4, 4], np.float32), W._identity34(), 0.0,
                     np.array([2], np.int32), np.array([[L2, 0, 0, 0.1]], np.float32), np.zeros((0, 2), np.int32))
    for q1, q2 in [(0.1, 0.2), (-1.0, 2.0), (3.0, -0.5)]:
        c = O.fk(m, [q1, q2])[0]
        np.testing.assert_allclose(c, [L1 * math.cos(q1) + L2 * math.cos(q1 + q2),
                                       L1 * math.sin(q1) + L2 * math.sin(q1 + q2), 0.0], atol=1e-7)


def test_fk_point_robot_and_base():
    m = W.disc_robot(0.25, 0.1)
    np.testing.assert_allclose(O.fk(m, [3.0, 4.0])[0], [3.0, 4.0, np.float32(0.1)], atol=1e-12)
    yaw = 0.6
    m.base = W._pose(1.0, 2.0, 0.5, yaw)
    m.sphere_xyzr = np.array([[0.1, 0.0, 0.0, 0.2]], np.float32)
    c = O.fk(m, [0.0, 0.0])[0]
    cy, sy = float(np.float32(math.cos(yaw))), float(np.float32(math.sin(yaw)))
    np.testing.assert_allclose(c, [1.0 + cy * 0.1, 2.0 + sy * 0.1, 0.5 + np.float32(0.1)], atol=1e-7)
    m3 = copy.deepcopy(m)
    m3.dof = 3
    m3.base = W._identity34()
    m3.sphere_xyzr = np.array([[0.0, 0.0, 0.0, 0.2]], np.float32)
    np.testing.assert_allclose(O.fk(m3, [1.0, -2.0, 0.7])[0], [1.0, -2.0, 0.7], atol=1e-12)


def test_fk_panda_zero_pose():
    g = json.loads((GOLD / "panda_zero_pose.json").read_text())
    m = W.panda_like(W._identity34(), None)
    links = sorted(int(k) for k in g["frames"])
    m.sphere_link = np.array(links, np.int32)
    m.sphere_xyzr = np.zeros((len(links), 4), np.float32)
    c = O.fk(m, np.zeros(7))
    for k, row in zip(links, c):
        np.testing.assert_allclose(row, g["frames"][str(k)], atol=g["tol"])


# --------------------------------------------------------------------------- CC

def test_sphere_box_cases():
    box = [0.0, 0.0, 0.0, 1.0, 2.0, 3.0]
    r = 0.25
    assert O.sphere_box([0.5, 1.0, 1.5], r, box) == pytest.approx(-r)          # inside
    assert O.sphere_box([1.0, 1.0, 1.5], r, box) == pytest.approx(-r)          # on a face
    assert O.sphere_box([1.5, 1.0, 1.5], r, box) == pytest.approx(0.5 - r)     # off a face
    assert O.sphere_box([1.3, 2.4, 1.5], r, box) == pytest.approx(0.5 - r)     # off an edge (0.3, 0.4)
    assert O.sphere_box([-0.1, -0.2, -0.2], r, box) == pytest.approx(0.3 - r)  # off a corner
    assert O.sphere_box([-1.0, 1.0, 1.5], r, box) == pytest.approx(1.0 - r)


def test_sphere_sphere_345():
    assert O.sphere_sphere([0, 0, 0], 0.5, [3, 4, 0], 1.0) == pytest.approx(3.5)
    assert O.sphere_sphere([1, 1, 1], 1.0, [1, 1, 1.5], 0.2) == pytest.approx(-0.7)


# --------------------------------------------------------------- discretisation

def _disc_query(s0, g0, s1, g1, T=None, res=0.05, r=0.25):
    models = [W.disc_robot(r), W.disc_robot(r)]
    bb = W.BatchBuilder(2, T is not None)
    steps = None if T is None else [[T], [T]]
    bb.add([0, 1], [np.array([s0, g0]), np.array([s1, g1])], steps)
    return W.Workload("discs", models, [], bb.build(res), env=-1, check_env=False)


def test_steps_from_resolution():
    cases = [(((0, 0), (1, 0)), 20), (((0, 0), (1.01, 0)), 21), (((2, 2), (2, 2)), 0),
             (((0, 0), (3, 4)), 100)]
    for (s, g), T in cases:
        w = _disc_query(s, g, (5, 5), (5, 5))
        assert O.Oracle(w).query_T()[0] == T
    # the composite motion takes the longest robot's duration (Sec. IV-A3)
    w = _disc_query((0, 0), (1, 0), (5, 5), (5, 7))
    assert O.Oracle(w).query_T()[0] == 40
    # joint space: |dq| = 0.5 rad at 1/32 rad per step is exactly 16 steps
    arm = W.panda_like(W._identity34(), None)
    bb = W.BatchBuilder(7, False)
    a = np.zeros(7, np.float32)
    b = a.copy()
    b[2] = 0.5
    bb.add([0], [np.array([a, b])])
    assert O.Oracle(W.Workload("a", [arm], [], bb.build(1 / 32), -1, False)).query_T()[0] == 16


# ---------------------------------------------------------- closed-form discs

def _disc_closed_form(s0, g0, s1, g1, T, R):
    p0 = np.subtract(s1, s0, dtype=np.float64)
    v = np.subtract(g1, s1, dtype=np.float64) - np.subtract(g0, s0, dtype=np.float64)
    A, B, Cc = v @ v, 2 * p0 @ v, p0 @ p0 - R * R
    first = -1
    disc = B * B - 4 * A * Cc
    if A > 0 and disc > 0:
        t1 = (-B - math.sqrt(disc)) / (2 * A)
        t2 = (-B + math.sqrt(disc)) / (2 * A)
        # smallest integer t in [0, T] with t1 < t/T < t2
        cand = max(0, math.floor(t1 * T) + 1)
        if cand <= T and cand / T < t2:
            first = cand
        near = min(abs(t1 * T - round(t1 * T)), abs(t2 * T - round(t2 * T)))
    elif A == 0:
        first = 0 if Cc < 0 else -1
        near = 1.0
    else:
        near = 1.0
    tau = 0.0 if A == 0 else min(1.0, max(0.0, -(p0 @ v) / A))
    dmin = float(np.linalg.norm(p0 + v * tau)) - R
    return first, near, dmin, math.sqrt(A)


def test_closed_form_linear_discs():
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(400):
        s0, g0, s1, g1 = (rng.uniform(0, 4, 2).astype(np.float32) for _ in range(4))
        T = int(rng.integers(5, 120))
        first, near, dmin, speed = _disc_closed_form(s0, g0, s1, g1, T, 0.5)
        if near < 1e-6:
            continue
        w = _disc_query(s0, g0, s1, g1, T=T)
        o = O.Oracle(w)
        f = o.ffc()[0]
        assert f[0] == first
        if first >= 0:
            assert tuple(f[1:]) == (0, 1)
        assert bool(o.mv(check_env=False)[0]) == (first < 0)
        sampled = o.mv_min_clearance(check_env=False)[0]
        assert dmin - 1e-9 <= sampled <= dmin + speed / (2 * T) + 1e-9
        checked += 1
    assert checked > 350


def test_head_on_golden():
    g = json.loads((GOLD / "head_on_discs.json").read_text())
    for key in ("crossing", "apart"):
        c = g[key]
        w = _disc_query(c["s0"], c["g0"], c["s1"], c["g1"], T=g["T"], r=g["radius"])
        o = O.Oracle(w)
        assert list(o.ffc()[0]) == c["ffc"]
        assert bool(o.mv(check_env=False)[0]) == c["mv"]
        if "conflict_states" in c:
            conf = [t for t in range(g["T"] + 1) if o.pair_clearances(0, t)[0] < 0]
            assert conf == c["conflict_states"]


# ------------------------------------------------------------- paper lane maps

def test_fig2_rake_and_linear_maps():
    g = json.loads((GOLD / "fig2_rake_example.json").read_text())
    for c in g["cases"]:
        assert BF.rake(c["t_total"], c["W"], c["b"]) == c["rake"]
        assert BF.linear(c["t_total"], c["W"], c["b"]) == c["linear"]
    # every timestep is covered exactly once by the rake batches
    for tt in (1, 7, 32, 33, 100):
        for Wd in (1, 4, 8, 32):
            nb = math.ceil(tt / Wd)
            seen = sorted(t for b in range(nb) for t in BF.rake(tt, Wd, b))
            assert seen == list(range(tt))


# --------------------------------------------------- brute force on tiny inputs

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("timed", [True, False])
def test_bruteforce_tiny(seed, timed):
    w = tiny_workload(100 + seed, n_queries=10, timed=timed)
    o = O.Oracle(w)
    mv = o.mv()
    mv_noenv = o.mv(check_env=False)
    ffc = o.ffc()
    T = o.query_T()
    for q in range(w.batch.n_queries):
        g = BF.Geometry(w, q)
        assert g.T == T[q]
        conf = BF.all_conflicts(g)
        exp_ffc = min(conf) if conf else (-1, -1, -1)
        assert tuple(ffc[q]) == exp_ffc
        assert bool(mv_noenv[q]) == (not conf)
        assert bool(mv[q]) == (not conf and not BF.any_env(g))
        for Wd in (1, 4, 8, 32):
            assert BF.ffc_alg2(g, Wd) == exp_ffc
            for hier in (False, True):
                for pack in ("rake", "linear"):
                    assert BF.mv_alg1(g, Wd, hier, True, pack) == bool(mv[q])
                    assert BF.mv_alg1(g, Wd, hier, False, pack) == bool(mv_noenv[q])


# ------------------------------------------------------------------ invariants

def _permute(w, q, perm):
    b = w.batch
    s0 = b.q_robot_off[q]
    bb = W.BatchBuilder(b.wp_stride, b.seg_steps is not None)
    robots, paths, steps = [], [], []
    for k in perm:
        s = s0 + k
        w0, w1 = b.slot_wp_off[s], b.slot_wp_off[s + 1]
        robots.append(int(b.slot_robot[s]))
        paths.append(b.waypoints[w0:w1])
        if b.seg_steps is not None:
            steps.append(b.seg_steps[w0:w1 - 1])
    bb.add(robots, paths, steps if b.seg_steps is not None else None, 0, w.env)
    return W.Workload("perm", w.models, w.envs, bb.build(b.resolution), w.env, w.check_env)


def _reverse(w, q):
    b = w.batch
    bb = W.BatchBuilder(b.wp_stride, b.seg_steps is not None)
    robots, paths, steps = [], [], []
    T = BF.composite_T(w, q)
    for s in range(b.q_robot_off[q], b.q_robot_off[q + 1]):
        w0, w1 = b.slot_wp_off[s], b.slot_wp_off[s + 1]
        robots.append(int(b.slot_robot[s]))
        P = b.waypoints[w0:w1][::-1]
        if b.seg_steps is not None:
            st = list(b.seg_steps[w0:w1 - 1][::-1])
            pad = T - sum(st)   # a shorter path holds its end: reversed, it waits at the start
            if pad > 0:
                P = np.concatenate([P[:1], P])
                st = [pad] + st
            steps.append(st)
        paths.append(P)
    bb.add(robots, paths, steps if b.seg_steps is not None else None, 0, w.env)
    return W.Workload("rev", w.models, w.envs, bb.build(b.resolution), w.env, w.check_env)


@pytest.mark.parametrize("seed", range(4))
def test_invariants_permutation_reversal(seed):
    w = tiny_workload(200 + seed, n_queries=10, timed=bool(seed % 2))
    o = O.Oracle(w)
    mv, ffc = o.mv(), o.ffc()
    rng = np.random.default_rng(seed)
    for q in range(w.batch.n_queries):
        n = int(w.batch.q_robot_off[q + 1] - w.batch.q_robot_off[q])
        perm = rng.permutation(n)
        wp = _permute(w, q, perm)
        op = O.Oracle(wp)
        assert op.mv()[0] == mv[q]
        fp = op.ffc()[0]
        assert fp[0] == ffc[q][0]
        if fp[0] >= 0:   # the permuted pair is a conflicting pair of the original at t*
            i, j = sorted((perm[fp[1]], perm[fp[2]]))
            pc = o.pair_clearances(q, fp[0])
            k = i * n - i * (i + 1) // 2 + (j - i - 1)
            assert pc[k] < 0
        wr = _reverse(w, q)
        assert O.Oracle(wr).mv()[0] == mv[q]


@pytest.mark.parametrize("seed", range(4))
def test_invariants_env_padding(seed):
    w = tiny_workload(300 + seed, n_queries=12, timed=True)
    o = O.Oracle(w)
    ffc = o.ffc()
    # FFC never looks at obstacles
    w2 = copy.copy(w)
    w2.batch = copy.copy(w.batch)
    w2.batch.q_env = np.full(w.batch.n_queries, -1, np.int32)
    w2.env = -1
    np.testing.assert_array_equal(O.Oracle(w2).ffc(), ffc)
    # MV without environment is false exactly when FFC finds a conflict
    np.testing.assert_array_equal(o.mv(check_env=False) == 0, ffc[:, 0] >= 0)
    # more checks can only invalidate
    assert np.all(o.mv() <= o.mv(check_env=False))
    # padding: holding the last configuration == an explicit stationary segment
    T = o.query_T()
    b = w.batch
    for q in range(b.n_queries):
        bb = W.BatchBuilder(b.wp_stride, True)
        robots, paths, steps = [], [], []
        for s in range(b.q_robot_off[q], b.q_robot_off[q + 1]):
            w0, w1 = b.slot_wp_off[s], b.slot_wp_off[s + 1]
            P = b.waypoints[w0:w1]
            st = list(b.seg_steps[w0:w1 - 1])
            pad = int(T[q] - sum(st))
            if pad > 0:
                P = np.concatenate([P, P[-1:]])
                st.append(pad)
            robots.append(int(b.slot_robot[s]))
            paths.append(P)
            steps.append(st)
        bb.add(robots, paths, steps, 0, w.env)
        wq = W.Workload("pad", w.models, w.envs, bb.build(), w.env, True)
        oq = O.Oracle(wq)
        assert oq.mv()[0] == o.mv([q])[0]
        np.testing.assert_array_equal(oq.ffc()[0], ffc[q])


def test_decidability_and_clearance_consistency():
    w = tiny_workload(400, n_queries=12, timed=True)
    o = O.Oracle(w)
    mv, mc = o.mv(), o.mv_min_clearance()
    assert np.all((mc < 0) == (mv == 0))
    for q in range(w.batch.n_queries):
        T = int(o.query_T([q])[0])
        ts = list(range(T + 1))
        per = o.clearance(q, ts)
        assert np.isclose(per.min(), mc[q]) or (np.isinf(per.min()) and np.isinf(mc[q]))
    # FFC decidability agrees with the pair clearances it summarises
    dec = o.ffc_decidable(margin=1e-4)
    ffc = o.ffc()
    for q in range(w.batch.n_queries):
        T = int(o.query_T([q])[0])
        vals = []
        for t in range(T + 1):
            for v in o.pair_clearances(q, t):
                vals.append(v)
                if v < 0:
                    break
            if vals and vals[-1] < 0:
                break
        exp = all(v > 1e-4 for v in vals[:-1]) and (vals[-1] < -1e-4 if ffc[q][0] >= 0 else (not vals or vals[-1] > 1e-4))
        assert bool(dec[q]) == bool(exp)


@pytest.mark.parametrize("seed", range(4))
def test_ffc_below_bruteforce(seed):
    """The first pair deeper than a bound (the test of undecidable FFC answers)
    against exhaustive enumeration of every (t, i, j) below the bound; bound 0
    is FFC itself, and a lower bound never comes earlier."""
    w = tiny_workload(450 + seed, n_queries=10, timed=bool(seed & 1), max_robots=4)
    o = O.Oracle(w)
    ffc = o.ffc()
    res = {b: o.ffc_below(b) for b in (0.03, 0.0, -1e-4, -0.02, -0.08)}
    np.testing.assert_array_equal(res[0.0], ffc)
    for q in range(w.batch.n_queries):
        g = BF.Geometry(w, q)
        for b, r in res.items():
            conf = BF.all_conflicts(g, b)
            assert tuple(r[q]) == (min(conf) if conf else (-1, -1, -1))
        keys = [tuple(res[b][q]) if res[b][q][0] >= 0 else (math.inf,) for b in (0.03, 0.0, -1e-4, -0.02, -0.08)]
        assert keys == sorted(keys)


def test_ffc_below_closed_form_discs():
    """Two linearly moving discs of radius 0.25: the pair clearance is below b
    exactly when the centers are closer than 0.5 + b, so the first such state
    is the closed-form first conflict with R = 0.5 + b."""
    rng = np.random.default_rng(17)
    checked = 0
    for _ in range(300):
        s0, g0, s1, g1 = (rng.uniform(0, 4, 2).astype(np.float32) for _ in range(4))
        T = int(rng.integers(5, 120))
        b = float(rng.choice([-0.1, -1e-4, 0.05]))
        first, near, _, _ = _disc_closed_form(s0, g0, s1, g1, T, 0.5 + b)
        if near < 1e-6:
            continue
        f = O.Oracle(_disc_query(s0, g0, s1, g1, T=T)).ffc_below(b)[0]
        assert f[0] == first
        if first >= 0:
            assert tuple(f[1:]) == (0, 1)
        checked += 1
    assert checked > 250


def test_ffc_below_equals_ffc_of_shrunk_spheres():
    """Clearance below -m is a collision of the same spheres with every
    radius reduced by m/2: the first deep conflict is FFC of the shrunk
    robots."""
    m = 0.04
    w = tiny_workload(470, n_queries=16, timed=True, max_robots=4)
    shrunk = copy.deepcopy(w)
    for mdl in shrunk.models:
        mdl.sphere_xyzr[:, 3] = (mdl.sphere_xyzr[:, 3].astype(np.float64) - m / 2).astype(np.float32)
    assert all(float(mdl.sphere_xyzr[:, 3].min()) > 0 for mdl in shrunk.models)
    np.testing.assert_array_equal(O.Oracle(w).ffc_below(-m), O.Oracle(shrunk).ffc())


def test_ffc_tie_is_lexicographic():
    """Alg. 2 keeps the earliest pair on ties (strict comparison, i-major
    loops): at t = 0 both (0,3) and (1,2) overlap, (0,3) comes first."""
    models = [W.disc_robot(0.25) for _ in range(4)]
    bb = W.BatchBuilder(2, True)
    pos = [(0.0, 0.0), (5.0, 0.0), (5.3, 0.0), (0.3, 0.0)]
    bb.add([0, 1, 2, 3], [np.array([p, p]) for p in pos], [[3]] * 4)
    w = W.Workload("tie", models, [], bb.build(), -1, False)
    assert list(O.Oracle(w).ffc()[0]) == [0, 0, 3]


@pytest.mark.parametrize("seed", range(3))
def test_bruteforce_many_robots(seed):
    w = tiny_workload(500 + seed, n_queries=6, timed=True, max_robots=5, max_steps=3)
    o = O.Oracle(w)
    ffc = o.ffc()
    for q in range(w.batch.n_queries):
        g = BF.Geometry(w, q)
        conf = BF.all_conflicts(g)
        assert tuple(ffc[q]) == (min(conf) if conf else (-1, -1, -1))
        assert BF.ffc_alg2(g, 4) == tuple(ffc[q])


@pytest.mark.parametrize("seed", range(2))
def test_bruteforce_large_teams(seed):
    """Teams of 9-16 robots (up to 120 pairs, pair indices past 31): the
    oracle's FFC against every conflict enumerated and against Alg. 2 with
    lane batches of 4, and its MV against Alg. 1 restated."""
    w = tiny_workload(520 + seed, n_queries=4, timed=True, min_robots=9, max_robots=16, max_steps=2,
                      n_models=3)
    o = O.Oracle(w)
    ffc = o.ffc()
    mv = o.mv()
    seen_high = False
    for q in range(w.batch.n_queries):
        g = BF.Geometry(w, q)
        conf = BF.all_conflicts(g)
        assert tuple(ffc[q]) == (min(conf) if conf else (-1, -1, -1))
        assert BF.ffc_alg2(g, 4) == tuple(ffc[q])
        assert bool(mv[q]) == BF.mv_alg1(g, 4, hierarchical=False, check_env=True)
        seen_high |= any(j >= 8 for _, _, j in conf)
    assert seen_high


# ------------------------------------------- prioritized planner's MV variant

def _discs_timed(paths, T, r=0.25, env=None):
    """n disc robots, each on a straight timed motion of T steps."""
    models = [W.disc_robot(r) for _ in paths]
    bb = W.BatchBuilder(2, True)
    bb.add(list(range(len(paths))), [np.array([s, g], np.float32) for s, g in paths], [[T]] * len(paths),
           0, -1 if env is None else 0)
    return W.Workload("discs", models, [] if env is None else [env], bb.build(0.05),
                      env=-1 if env is None else 0, check_env=env is not None)


def test_prio_closed_form_discs():
    """Three discs on straight lines: the prioritized MV is invalid exactly
    when disc 0 meets disc 1 or disc 2 (closed-form time of closest approach);
    a meeting of discs 1 and 2 alone leaves it valid.  The full MV needs all
    three pairs apart."""
    rng = np.random.default_rng(31)
    checked = seen_12_only = 0
    for _ in range(300):
        p = [tuple(rng.uniform(0, 4, 2).astype(np.float32) for _ in range(2)) for _ in range(3)]
        T = int(rng.integers(5, 80))
        cf = {}
        for i, j in ((0, 1), (0, 2), (1, 2)):
            cf[i, j] = _disc_closed_form(p[i][0], p[i][1], p[j][0], p[j][1], T, 0.5)
        if min(c[1] for c in cf.values()) < 1e-6:
            continue
        w = _discs_timed(p, T)
        o = O.Oracle(w)
        prio_valid = cf[0, 1][0] < 0 and cf[0, 2][0] < 0
        assert bool(o.mv(priority=True)[0]) == prio_valid
        assert bool(o.mv()[0]) == (prio_valid and cf[1, 2][0] < 0)
        lo = min(cf[0, 1][2], cf[0, 2][2])
        hi = min(cf[k][2] + cf[k][3] / (2 * T) for k in ((0, 1), (0, 2)))
        assert lo - 1e-9 <= o.mv_min_clearance(priority=True)[0] <= hi + 1e-9
        seen_12_only += prio_valid and cf[1, 2][0] >= 0
        checked += 1
    assert checked > 250 and seen_12_only > 5


def test_prio_obstacles_of_current_robot_only():
    """With obstacles, only disc 0's contacts count: a box on disc 1's path
    leaves the prioritized MV valid, the same box on disc 0's path does not."""
    box = W.Env(np.zeros((0, 4), np.float32), np.array([[1.8, 1.8, -1.0, 2.2, 2.2, 1.0]], np.float32), "box")
    through, aside = ((0.5, 2.0), (3.5, 2.0)), ((0.5, 5.0), (3.5, 5.0))
    far = ((7.0, 8.0), (9.0, 8.0))
    o = O.Oracle(_discs_timed([aside, through, far], 40, env=box))
    assert bool(o.mv(priority=True)[0]) and not bool(o.mv()[0])
    o = O.Oracle(_discs_timed([through, aside, far], 40, env=box))
    assert not bool(o.mv(priority=True)[0]) and not bool(o.mv()[0])
    assert bool(o.mv(priority=True, check_env=False)[0])


@pytest.mark.parametrize("seed", range(4))
def test_prio_bruteforce_tiny(seed):
    """The prioritized MV against Alg. 1 as Sec. IV-C modifies it, restated in
    paper order with every lane width and packing, and its invariants: it
    only drops checks (full valid => prioritized valid), equals the full MV
    for two robots without obstacles, and does not depend on the order of the
    higher-priority robots."""
    w = tiny_workload(700 + seed, n_queries=10, timed=bool(seed % 2), max_robots=4)
    o = O.Oracle(w)
    full, full_ne = o.mv(), o.mv(check_env=False)
    pr, pr_ne = o.mv(priority=True), o.mv(priority=True, check_env=False)
    rng = np.random.default_rng(seed)
    for q in range(w.batch.n_queries):
        g = BF.Geometry(w, q)
        for Wd in (1, 8, 32):
            for pack in ("rake", "linear"):
                assert BF.mv_alg1_prio(g, Wd, True, pack) == bool(pr[q])
                assert BF.mv_alg1_prio(g, Wd, False, pack) == bool(pr_ne[q])
        assert pr[q] >= full[q] and pr_ne[q] >= full_ne[q]
        n = len(g.slots)
        if n == 2:
            assert pr_ne[q] == full_ne[q]
        if n >= 3:
            perm = [0] + list(rng.permutation(np.arange(1, n)))
            wp = _permute(w, q, perm)
            assert O.Oracle(wp).mv(priority=True)[0] == pr[q]


# ------------------------------------------------------- cylinder obstacles

CYL = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 2.0, 1.0])   # axis z in [0, 2], radius 1


@pytest.mark.parametrize("c, dist", [
    ((0.0, 0.0, 1.0), 0.0),        # on the axis, inside
    ((0.6, 0.0, 0.3), 0.0),        # inside, off the axis
    ((3.0, 0.0, 1.0), 2.0),        # beside the side wall
    ((0.0, 0.0, 5.0), 3.0),        # above the top cap, within the radius
    ((0.5, 0.0, -2.0), 2.0),       # below the bottom cap, within the radius
    ((4.0, 0.0, 6.0), 5.0),        # beyond the rim: 3-4-5 to the top edge
    ((0.0, -2.0, -3.0), math.hypot(1.0, 3.0)),   # beyond the bottom rim
    ((1.0, 0.0, 1.0), 0.0),        # on the side wall
])
def test_sphere_cylinder_cases(c, dist):
    assert O.sphere_cylinder(c, 0.25, CYL) == pytest.approx(dist - 0.25, abs=1e-12)


def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_sphere_cylinder_rigid_motion_and_ends():
    """A rigid motion of sphere and cylinder keeps the clearance; swapping
    the axis ends keeps it; a longer axis only adds clearance beyond the caps."""
    rng = np.random.default_rng(12)
    for _ in range(200):
        Rm, tr = _rotation(rng), rng.normal(size=3)
        c = rng.uniform(-3, 3, 3)
        r = rng.uniform(0, 0.5)
        ref = O.sphere_cylinder(c, r, CYL)
        a, b = Rm @ CYL[:3] + tr, Rm @ CYL[3:6] + tr
        moved = np.concatenate([a, b, [CYL[6]]])
        assert O.sphere_cylinder(Rm @ c + tr, r, moved) == pytest.approx(ref, abs=2e-6)
        swapped = np.concatenate([b, a, [CYL[6]]])
        assert O.sphere_cylinder(Rm @ c + tr, r, swapped) == pytest.approx(ref, abs=2e-6)


def test_sphere_cylinder_surface_sampling():
    """Outside the solid, the distance is the minimum over its surface: a dense
    sampling of the side wall and both caps bounds it from above and, to the
    sampling step, from below; inside, the distance is 0."""
    rng = np.random.default_rng(13)
    for _ in range(20):
        a = rng.uniform(-1, 1, 3)
        b = a + rng.normal(size=3)
        rho = rng.uniform(0.1, 0.8)
        cyl = np.concatenate([a, b, [rho]]).astype(np.float32).astype(np.float64)
        a, b, rho = cyl[:3], cyl[3:6], cyl[6]
        L = np.linalg.norm(b - a)
        u = (b - a) / L
        e1 = np.cross(u, [1.0, 0, 0] if abs(u[0]) < 0.9 else [0, 1.0, 0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(u, e1)
        ang = np.linspace(0, 2 * np.pi, 181)[:-1]
        ring = np.cos(ang)[:, None] * e1 + np.sin(ang)[:, None] * e2
        side = (a + np.linspace(0, L, 81)[:, None, None] * u + rho * ring[None]).reshape(-1, 3)
        disc = (np.linspace(0, rho, 21)[:, None, None] * ring[None]).reshape(-1, 3)
        surf = np.concatenate([side, a + disc, b + disc])
        step = max(2 * np.pi * rho / 180, L / 80, rho / 20)
        for _ in range(30):
            c = a + rng.uniform(-2.5, 2.5, 3)
            d = O.sphere_cylinder(c, 0.0, cyl)
            s, w = (c - a) @ u, c - a
            inside = 0 <= s <= L and np.linalg.norm(w - s * u) <= rho
            if inside:
                assert d == 0.0
                continue
            m = np.linalg.norm(surf - c, axis=1).min()
            assert d <= m + 1e-9 and d >= m - step


def test_disc_past_vertical_cylinder():
    """A disc moving in the plane z = 0 past a vertical cylinder through that
    plane: MV is invalid exactly when some sampled state brings the disc
    center within r + rho of the cylinder axis (planar distances, no oracle
    geometry)."""
    rng = np.random.default_rng(14)
    seen = [0, 0]
    for _ in range(300):
        cx, cy, rho = rng.uniform(2, 8), rng.uniform(2, 8), rng.uniform(0.2, 1.0)
        cyl = np.array([[cx, cy, -1.0, cx, cy, 1.0, rho]], np.float32)
        env = W.Env(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), "cyl", cyl)
        s, g = rng.uniform(0, 10, 2).astype(np.float32), rng.uniform(0, 10, 2).astype(np.float32)
        T = int(rng.integers(5, 80))
        w = _discs_timed([(s, g)], T, env=env)
        st = np.array([s + (g.astype(np.float64) - s) * (t / T) for t in range(T + 1)])
        d = np.linalg.norm(st - np.array([cx, cy], np.float32).astype(np.float64), axis=1) - 0.25 - float(cyl[0, 6])
        if np.abs(d).min() < 1e-6:
            continue
        expect = bool((d >= 0).all())
        assert bool(O.Oracle(w).mv()[0]) == expect
        # distance to the solid is 0 inside it, so the clearance is at least -r
        clr = np.maximum(d + 0.25, 0.0) - 0.25
        assert O.Oracle(w).mv_min_clearance()[0] == pytest.approx(clr.min(), abs=1e-6)
        seen[expect] += 1
    assert min(seen) > 20


@pytest.mark.parametrize("seed", range(3))
def test_bruteforce_tiny_cylinders(seed):
    """Random scenes with obstacle cylinders: the oracle's MV against a numpy
    restatement of the definition (its own cylinder distance), with and
    without the other obstacles' share of collisions."""
    w = tiny_workload(1300 + seed, n_queries=12, timed=bool(seed % 2), cylinders=5)
    only = copy.deepcopy(w)   # the same scene with the cylinders as the only obstacles
    only.envs[0].spheres = np.zeros((0, 4), np.float32)
    only.envs[0].aabbs = np.zeros((0, 6), np.float32)
    for ww, need in ((w, 2), (only, 2)):
        mv = O.Oracle(ww).mv()
        n_env = 0
        for q in range(ww.batch.n_queries):
            g = BF.Geometry(ww, q)
            conf = BF.all_conflicts(g)
            env = BF.any_env(g)
            assert bool(mv[q]) == (not conf and not env)
            n_env += env
        assert n_env >= need
