"""Seeded tiny random workloads for brute-force pins and edge-case parity.

Draws inputs only: point robots (dof 2 and 3) and short modified-DH chains
(dof 1-3) with 1-4 spheres, a handful of obstacle spheres and boxes, and
queries of 1-3 robots in start/goal or timed-waypoint form with ragged path
lengths (so padding is exercised).  The scale (about 2 m) makes roughly half
of the states collide.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2604_23960_gb300 import workloads as W


def _rand_pose(rng, span=1.0):
    yaw = rng.uniform(-math.pi, math.pi)
    x, y = rng.uniform(-span, span, 2)
    return W._pose(x, y, rng.uniform(-0.2, 0.2), yaw)


def random_robot(rng, kind=None):
    kind = rng.integers(0, 3) if kind is None else kind
    m = int(rng.integers(1, 5))
    xyzr = np.zeros((m, 4), np.float32)
    xyzr[:, :3] = rng.uniform(-0.15, 0.15, (m, 3))
    xyzr[:, 3] = rng.uniform(0.05, 0.25, m)
    if kind in (0, 1):   # point robot, dof 2 (fixed z) or dof 3
        dof = 2 if kind == 0 else 3
        links = rng.integers(0, 2, m).astype(np.int32)
        links[0] = 1
        return W.RobotModel(W.KIND_POINT, dof, np.zeros((dof, 4), np.float32), None,
                            np.full(dof, -1.0, np.float32), np.full(dof, 1.0, np.float32), _rand_pose(rng),
                            float(rng.uniform(-0.2, 0.2)), links, xyzr, np.zeros((0, 2), np.int32))
    dof = int(rng.integers(1, 4))
    dh = np.zeros((dof, 4), np.float32)
    dh[:, 0] = rng.uniform(0.0, 0.5, dof)
    dh[:, 1] = rng.choice([0.0, math.pi / 2, -math.pi / 2, rng.uniform(-3, 3)], dof)
    dh[:, 2] = rng.uniform(0.0, 0.4, dof)
    dh[:, 3] = rng.uniform(-1.0, 1.0, dof)
    flange = None if rng.uniform() < 0.5 else _rand_pose(rng, 0.2)
    links = rng.integers(0, dof + 2, m).astype(np.int32)
    xyzr[:, :3] += np.array([0.2, 0.0, 0.0], np.float32)
    pairs = [(a, b) for a in range(m) for b in range(a + 1, m) if links[a] != links[b] and rng.uniform() < 0.5]
    return W.RobotModel(W.KIND_DH, dof, dh, flange, np.full(dof, -math.pi, np.float32),
                        np.full(dof, math.pi, np.float32), _rand_pose(rng), 0.0, links, xyzr,
                        np.array(pairs, np.int32).reshape(-1, 2))


def random_env(rng, n_s=3, n_b=3, n_c=0):
    sph = np.zeros((n_s, 4), np.float32)
    sph[:, :3] = rng.uniform(-1.5, 1.5, (n_s, 3))
    sph[:, 3] = rng.uniform(0.05, 0.3, n_s)
    c = rng.uniform(-1.5, 1.5, (n_b, 3))
    h = rng.uniform(0.05, 0.3, (n_b, 3))
    env = W.Env(sph, np.concatenate([c - h, c + h], axis=1).astype(np.float32))
    if n_c:
        a = rng.uniform(-1.5, 1.5, (n_c, 3))
        d = rng.normal(size=(n_c, 3))
        d *= rng.uniform(0.2, 1.0, (n_c, 1)) / np.linalg.norm(d, axis=1, keepdims=True)
        env.cylinders = np.concatenate([a, a + d, rng.uniform(0.03, 0.25, (n_c, 1))], axis=1).astype(np.float32)
    return env


def random_config(rng, m: W.RobotModel):
    if m.kind == W.KIND_POINT:
        return rng.uniform(-1.0, 1.0, m.dof)
    return rng.uniform(-math.pi, math.pi, m.dof)


def tiny_workload(seed: int, n_queries: int = 12, timed: bool = True, max_robots: int = 3,
                  n_models: int = 5, max_steps: int = 6, resolution: float = 0.4, env: bool = True,
                  cylinders: int = 0, min_robots: int = 1):
    rng = np.random.default_rng(seed)
    models = [random_robot(rng) for _ in range(n_models)]
    envs = [random_env(rng, n_c=cylinders)] if env else []
    bb = W.BatchBuilder(3, timed)
    for _ in range(n_queries):
        n = int(rng.integers(min_robots, max_robots + 1))
        robots = [int(rng.integers(0, n_models)) for _ in range(n)]
        paths, steps = [], []
        for r in robots:
            if timed:
                k = int(rng.integers(1, 4))
                paths.append(np.array([random_config(rng, models[r]) for _ in range(k)]))
                steps.append(rng.integers(1, max_steps + 1, k - 1))
            else:
                paths.append(np.array([random_config(rng, models[r]) for _ in range(2)]))
        bb.add(robots, paths, steps if timed else None, int(rng.integers(0, 2)), 0 if env else -1)
    return W.Workload(f"tiny{seed}", models, envs, bb.build(resolution), env=0 if env else -1, check_env=True)
