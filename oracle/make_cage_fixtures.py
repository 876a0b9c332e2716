"""Draws the seeded Panda-cage fixtures that need the method's arithmetic.

Writes ``tests/golden/cage_fixtures.npz`` with
  self_pairs     (k, 2) int32   self-collision sphere pairs of the Panda-like
                                model: spheres on bodies at least two apart in
                                the chain, at least 0.02 m apart in the
                                mid-range configuration, and colliding in at
                                most 5% of 256 uniformly drawn configurations
                                (pairs that overlap across a joint in most
                                poses are geometry artefacts, not checks);
  endpoint_pool  (4, 1024, 7)   per cage arm, configurations uniform in the
                 float32        joint limits that are env+self valid with at
                                least 1 mm clearance (the paper samples motions
                                with valid endpoints, Sec. IV-A1).
With --cage8 it writes ``tests/golden/cage8_fixtures.npz`` instead:
  endpoint_pool  (8, 1024, 7)   per arm of the floor- and ceiling-mounted
                 float32        8-arm team, configurations uniform in the joint
                                limits that are valid against the cylinder cage
                                and themselves with at least 1 mm clearance
                                (self pairs from cage_fixtures.npz).
With --cage16 it writes ``tests/golden/cage16_fixtures.npz``:
  endpoint_pool  (8, 1024, 7)   the same for arms 8..15 of the 16-arm team
                 float32        (arms 0..7 are the 8-arm team's and keep its
                                pools);
  team_states    (256, 16, 7)   16-arm configurations valid as a whole (every
                 float32        arm env+self valid and clear of every other
                                arm by at least 1 mm), built arm by arm: arm k
                                takes the first of 32 pool draws that keeps
                                the configuration valid; configurations with
                                no such draw are dropped (random independent
                                endpoints of 16 crowded arms almost always
                                collide at once, while a planner's edges join
                                valid configurations).
Only the FP64 oracle evaluates geometry here.  Seeds: 301 (pair screening),
302 (endpoint pools), 303 (8-arm endpoint pools), 304 (16-arm endpoint pools),
305 (16-arm team configurations).
Usage: python oracle/make_cage_fixtures.py [--cage8 | --cage16]
"""
from __future__ import annotations

import os
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from paper_2604_23960_gb300 import workloads as W  # noqa: E402

OUT = ROOT / "tests" / "golden" / "cage_fixtures.npz"
OUT8 = ROOT / "tests" / "golden" / "cage8_fixtures.npz"
OUT16 = ROOT / "tests" / "golden" / "cage16_fixtures.npz"
POOL = 1024


def screen_self_pairs(seed: int = 301, n_cfg: int = 256, max_rate: float = 0.05, min_mid: float = 0.02):
    m = W.panda_like(W._identity34(), None)
    body = m.sphere_link
    r = m.sphere_xyzr[:, 3].astype(np.float64)
    cand = [(a, b) for a in range(m.n_spheres) for b in range(a + 1, m.n_spheres)
            if abs(int(body[a]) - int(body[b])) >= 2]
    cand = np.array(cand, np.int64)
    qmid = (W.PANDA_LO.astype(np.float64) + W.PANDA_HI) / 2
    c = O.fk(m, qmid)
    d = np.linalg.norm(c[cand[:, 0]] - c[cand[:, 1]], axis=1) - r[cand[:, 0]] - r[cand[:, 1]]
    keep = d > min_mid
    rng = np.random.default_rng(seed)
    hits = np.zeros(len(cand))
    for _ in range(n_cfg):
        q = rng.uniform(W.PANDA_LO, W.PANDA_HI)
        c = O.fk(m, q)
        d = np.linalg.norm(c[cand[:, 0]] - c[cand[:, 1]], axis=1) - r[cand[:, 0]] - r[cand[:, 1]]
        hits += d < 0
    keep &= hits / n_cfg <= max_rate
    return cand[keep].astype(np.int32)


def endpoint_pools(self_pairs, seed: int = 302, pool: int = POOL, chunk: int = 4096, arms=None, env=None,
                   first: int = 0):
    fx = {"self_pairs": self_pairs}
    arms = W.cage_arms(fx) if arms is None else arms
    env = W.cage_env() if env is None else env
    rng = np.random.default_rng(seed)
    pools = []
    threads = os.cpu_count() or 1
    for k in range(first, len(arms)):
        got = []
        while sum(len(g) for g in got) < pool:
            cfg = rng.uniform(W.PANDA_LO, W.PANDA_HI, (chunk, 7)).astype(np.float32)
            wps = np.repeat(cfg, 2, axis=0)       # start = goal: a single state
            b = W._fast_batch(chunk, 1, np.full(chunk, k, np.int32), wps, None, 1.0 / 32, W.KIND_MV, 0)
            wl = W.Workload("pool", arms, [env], b, env=0, check_env=True)
            m = O.Oracle(wl).mv_min_clearance(stop_below=-1.0, threads=threads)
            got.append(cfg[m > 1e-3])
        pools.append(np.concatenate(got)[:pool])
    return np.stack(pools).astype(np.float32)


def main():
    sp = screen_self_pairs()
    pools = endpoint_pools(sp)
    OUT.parent.mkdir(parents=True, exist_ok=True)
    np.savez_compressed(OUT, self_pairs=sp, endpoint_pool=pools)
    print(f"wrote {OUT}: {len(sp)} self pairs, endpoint pools {pools.shape}")


def main_cage8():
    sp = W.load_cage_fixtures()["self_pairs"]
    pools = endpoint_pools(sp, seed=303, arms=W.cage8_arms({"self_pairs": sp}), env=W.cage_env_cyl())
    np.savez_compressed(OUT8, endpoint_pool=pools)
    print(f"wrote {OUT8}: endpoint pools {pools.shape}")


def team_states(arms, pools, env, n_states: int, seed: int, draws: int = 32, spare: int = 4):
    """Whole-team configurations built arm by arm from per-arm pools; the
    oracle's exhaustive minimum clearance (obstacles, self pairs, every robot
    pair) of each partial team must stay above 1 mm."""
    rng = np.random.default_rng(seed)
    n, P = len(arms), pools.shape[1]
    G = n_states * spare
    states = np.zeros((G, n, 7), np.float32)
    alive = np.ones(G, bool)
    threads = os.cpu_count() or 1
    for k in range(n):
        cand = pools[k][rng.integers(0, P, (G, draws))]          # (G, draws, 7)
        team = np.repeat(states[:, None, :k + 1], draws, axis=1)  # (G, draws, k+1, 7)
        team[:, :, k] = cand
        cfg = team.reshape(-1, k + 1, 7)
        wps = np.repeat(cfg.reshape(-1, 7), 2, axis=0)            # start = goal: one state
        nq = G * draws
        b = W._fast_batch(nq, k + 1, np.tile(np.arange(k + 1, dtype=np.int32), nq), wps, None, 1.0 / 32,
                          W.KIND_MV, 0)
        wl = W.Workload("team", arms[:k + 1], [env], b, env=0, check_env=True)
        ok = (O.Oracle(wl).mv_min_clearance(threads=threads) > 1e-3).reshape(G, draws)
        has = ok.any(axis=1)
        first = ok.argmax(axis=1)
        states[has, k] = cand[has, first[has]]
        alive &= has
    out = states[alive]
    if len(out) < n_states:
        raise RuntimeError(f"only {len(out)} team configurations of {n_states}")
    return out[:n_states]


def main_cage16():
    sp = W.load_cage_fixtures()["self_pairs"]
    arms = W.cage16_arms({"self_pairs": sp})
    env = W.cage_env_cyl()
    pools = endpoint_pools(sp, seed=304, arms=arms, env=env, first=8)
    allp = np.concatenate([W.load_cage8_fixtures()["endpoint_pool"], pools])
    team = team_states(arms, allp, env, 256, seed=305)
    np.savez_compressed(OUT16, endpoint_pool=pools, team_states=team)
    print(f"wrote {OUT16}: endpoint pools {pools.shape}, team states {team.shape}")


if __name__ == "__main__":
    if "--cage8" in sys.argv[1:]:
        main_cage8()
    elif "--cage16" in sys.argv[1:]:
        main_cage16()
    else:
        main()
