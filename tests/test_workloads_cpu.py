"""The seeded workloads keep the properties their generators state, checked
with the FP64 oracle on the CPU: the 16-arm team configurations are valid as
a whole and stay valid for the 4- and 8-arm subteams the validation study
uses, the 16-arm edges start valid and move no arm by more than 0.5 rad, and
the study's motions join two valid configurations."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2604_23960_gb300 import workloads as W


def _single_states(models, env, cfg):
    """A batch of one-state queries (start = goal) of len(models) robots."""
    nq, n = cfg.shape[0], cfg.shape[1]
    wps = np.repeat(cfg.reshape(-1, 7), 2, axis=0)
    b = W._fast_batch(nq, n, np.tile(np.arange(n, dtype=np.int32), nq), wps, None, 1.0 / 32, W.KIND_MV, 0)
    return W.Workload("states", models, [env], b, env=0, check_env=True)


def test_team_states_valid_for_every_subteam():
    fx = W.load_cage_fixtures()
    team = W.load_cage16_fixtures()["team_states"]
    arms = W.cage16_arms(fx)
    env = W.cage_env_cyl()
    idx = np.arange(0, team.shape[0], 8)             # 32 of the 256 configurations
    for n in (4, 8, 16):
        w = _single_states(arms[:n], env, team[idx, :n])
        m = O.Oracle(w).mv_min_clearance(threads=4)
        assert np.all(m > 1e-3), f"{n} arms: a configuration is not valid by 1 mm ({m.min()})"


def test_cage16_edges_start_valid_and_are_short():
    w = W.make_cage16_mv(64)
    b = w.batch
    wp = b.waypoints.reshape(-1, 2, b.wp_stride)[:, :, :7]   # per slot: start, goal
    step = np.linalg.norm(wp[:, 1] - wp[:, 0], axis=1).reshape(64, 16)
    assert np.all(step.max(axis=1) <= 0.5 + 1e-5)
    starts = wp[:, 0].reshape(64, 16, 7)
    ws = _single_states(w.models, w.envs[0], starts)
    assert np.all(O.Oracle(ws).mv_min_clearance(threads=4) > 1e-3)


def test_study_motions_join_valid_configurations():
    for n in (4, 8):
        w = W.make_cage_team_study(n, 24)
        b = w.batch
        wp = b.waypoints.reshape(-1, 2, b.wp_stride)[:, :, :7].reshape(24, n, 2, 7)
        for end in (0, 1):
            ws = _single_states(w.models, W.cage_env_cyl(), wp[:, :, end])
            assert np.all(O.Oracle(ws).mv_min_clearance(threads=4) > 1e-3)
