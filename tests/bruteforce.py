"""Brute-force and paper-order re-statements used to pin the oracle.

Geometry comes from the oracle's FK (pinned separately against closed forms);
what this module restates independently is the *control* of the method:
PackCfgBatch rake / linear lane maps (Sec. III-A, Fig. 2), Alg. 1 in its
combined and hierarchical orders with early termination, Alg. 2 with its
first-timestep early return and per-batch minimum, and a full enumeration of
every (t, i, j) conflict without any early exit.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O


def rake(t_total: int, W: int, b: int):
    nb = math.ceil(t_total / W)
    return [b + nb * k for k in range(W) if b + nb * k < t_total]


def linear(t_total: int, W: int, b: int):
    return [t for t in range(b * W, b * W + W) if t < t_total]


def composite_T(w, q):
    b = w.batch
    s0, s1 = b.q_robot_off[q], b.q_robot_off[q + 1]
    T = 0
    for s in range(s0, s1):
        w0, w1 = b.slot_wp_off[s], b.slot_wp_off[s + 1]
        if b.seg_steps is None:
            dof = w.models[b.slot_robot[s]].dof
            a = b.waypoints[w0, :dof].astype(np.float64)
            g = b.waypoints[w0 + 1, :dof].astype(np.float64)
            d = math.sqrt(float(np.sum((g - a) ** 2)))
            Ts = 0 if d == 0 else math.ceil(d / float(np.float32(b.resolution)))
        else:
            Ts = int(np.sum(b.seg_steps[w0:w1 - 1]))
        T = max(T, Ts)
    return T


def config(w, q, s, t, T):
    b = w.batch
    w0, w1 = b.slot_wp_off[s], b.slot_wp_off[s + 1]
    dof = w.models[b.slot_robot[s]].dof
    P = b.waypoints[w0:w1, :dof].astype(np.float64)
    if b.seg_steps is None:
        return P[0] if T == 0 else P[0] + (P[1] - P[0]) * (t / T)
    tau = 0
    for k in range(w1 - w0 - 1):
        n = int(b.seg_steps[w0 + k])
        if t < tau + n:
            return P[k] + (P[k + 1] - P[k]) * ((t - tau) / n)
        tau += n
    return P[-1]


class Geometry:
    """World sphere centers per (t, robot) of one query, from the oracle FK."""

    def __init__(self, w, q):
        self.w, self.q = w, q
        b = w.batch
        self.slots = list(range(b.q_robot_off[q], b.q_robot_off[q + 1]))
        self.models = [w.models[b.slot_robot[s]] for s in self.slots]
        self.T = composite_T(w, q)
        e = int(b.q_env[q]) if b.q_env is not None else w.env
        self.env = None if e < 0 else w.envs[e]
        self._c = {}

    def centers(self, t, i):
        key = (t, i)
        if key not in self._c:
            self._c[key] = O.fk(self.models[i], config(self.w, self.q, self.slots[i], t, self.T))
        return self._c[key]

    def pair_hit(self, t, i, j, bound=0.0):
        """Some sphere pair of robots i and j at state t has clearance below
        `bound` (0: they collide)."""
        ci, cj = self.centers(t, i), self.centers(t, j)
        ri = self.models[i].sphere_xyzr[:, 3].astype(np.float64)
        rj = self.models[j].sphere_xyzr[:, 3].astype(np.float64)
        d = np.linalg.norm(ci[:, None, :] - cj[None, :, :], axis=2) - ri[:, None] - rj[None, :]
        return bool((d < bound).any())

    def env_hit(self, t, i):
        c = self.centers(t, i)
        m = self.models[i]
        r = m.sphere_xyzr[:, 3].astype(np.float64)
        if self.env is not None:
            es = self.env.spheres.astype(np.float64)
            if len(es):
                d = np.linalg.norm(c[:, None, :] - es[None, :, :3], axis=2) - r[:, None] - es[None, :, 3]
                if (d < 0).any():
                    return True
            for bx in self.env.aabbs.astype(np.float64):
                e = np.maximum(np.maximum(bx[:3] - c, c - bx[3:]), 0.0)
                if ((np.linalg.norm(e, axis=1) - r) < 0).any():
                    return True
            for cy in np.asarray(getattr(self.env, "cylinders", np.zeros((0, 7)))).astype(np.float64):
                a, b, rho = cy[:3], cy[3:6], cy[6]
                L = np.linalg.norm(b - a)
                u = (b - a) / L
                s = (c - a) @ u
                d = np.linalg.norm(c - a - s[:, None] * u, axis=1)
                gap = np.hypot(np.maximum(np.maximum(-s, s - L), 0.0), np.maximum(d - rho, 0.0))
                if ((gap - r) < 0).any():
                    return True
        for a, bb in m.self_pairs.reshape(-1, 2):
            if np.linalg.norm(c[a] - c[bb]) - r[a] - r[bb] < 0:
                return True
        return False


def mv_alg1(g: Geometry, W: int, hierarchical: bool, check_env: bool, packing: str = "rake"):
    """Alg. 1 with the given lane width, order and packing; returns (valid, states_checked)."""
    tt = g.T + 1
    n = len(g.slots)
    pack = rake if packing == "rake" else linear
    nb = math.ceil(tt / W)
    if hierarchical and check_env:
        for b in range(nb):
            for i in range(n):
                for t in pack(tt, W, b):
                    if g.env_hit(t, i):
                        return False
    for b in range(nb):
        if not hierarchical and check_env:
            for i in range(n):
                for t in pack(tt, W, b):
                    if g.env_hit(t, i):
                        return False
        for i in range(n - 1):
            for j in range(i + 1, n):
                for t in pack(tt, W, b):
                    if g.pair_hit(t, i, j):
                        return False
    return True


def mv_alg1_prio(g: Geometry, W: int, check_env: bool, packing: str = "rake"):
    """Alg. 1 as the prioritized planner modifies it (Sec. IV-C, PP-ST-RRT):
    the robot loop of the obstacle / self step runs over the current robot
    (slot 0) only, and the robot-robot loop over the pairs of the current
    robot with each higher-priority robot (slots 1..n-1)."""
    tt = g.T + 1
    n = len(g.slots)
    pack = rake if packing == "rake" else linear
    for b in range(math.ceil(tt / W)):
        if check_env:
            for t in pack(tt, W, b):
                if g.env_hit(t, 0):
                    return False
        for j in range(1, n):
            for t in pack(tt, W, b):
                if g.pair_hit(t, 0, j):
                    return False
    return True


def ffc_alg2(g: Geometry, W: int):
    """Alg. 2: linear batches, return at a conflict on the batch's first
    timestep, otherwise the batch minimum over robot pairs (earliest pair on
    ties, by the strict comparison)."""
    tt = g.T + 1
    n = len(g.slots)
    nb = math.ceil(tt / W)
    for b in range(nb):
        t0 = b * W
        best = None
        for i in range(n - 1):
            for j in range(i + 1, n):
                tc = next((t for t in linear(tt, W, b) if g.pair_hit(t, i, j)), None)
                if tc is None:
                    continue
                if tc == t0:
                    return (tc, i, j)
                if best is None or best[0] > tc:
                    best = (tc, i, j)
        if best is not None:
            return best
    return (-1, -1, -1)


def all_conflicts(g: Geometry, bound=0.0):
    """Every colliding (t, i, j), exhaustive; with a bound, every (t, i, j)
    whose pair clearance is below it."""
    n = len(g.slots)
    return [(t, i, j) for t in range(g.T + 1) for i in range(n) for j in range(i + 1, n)
            if g.pair_hit(t, i, j, bound)]


def any_env(g: Geometry):
    return any(g.env_hit(t, i) for t in range(g.T + 1) for i in range(len(g.slots)))
