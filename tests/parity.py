"""Comparison rules between the CUDA path and the FP64 oracle.

MV booleans and FFC (t, i, j) triples must be identical on every query whose
oracle clearances keep a margin of 1e-4 m from zero (the FP32 kernel and the
FP64 oracle can only disagree on near-tangent contacts).  On the remaining
queries the GPU answer must be *consistent*: a reported collision has oracle
clearance below +1e-4, a reported valid motion has none below -1e-4, and an
FFC answer lies no later than the oracle's first pair deeper than -1e-4.
Clearance values must agree within 1e-5 m.
"""
from __future__ import annotations

import os

import numpy as np

MARGIN = 1e-4        # m: decidability margin on clearances
CLR_TOL = 1e-5       # m: absolute tolerance on clearance values
THREADS = os.cpu_count() or 1


def check_mv(o, gpu_valid, idx=None, check_env=True, margin=MARGIN, priority=False):
    """Returns (n_checked, n_undecidable).  priority: against the prioritized
    planner's MV (slot 0 against the obstacles, itself and slots 1..n-1)."""
    n = o.w.batch.n_queries
    idx = np.arange(n) if idx is None else np.asarray(idx)
    g = np.asarray(gpu_valid)[idx].astype(bool) if len(gpu_valid) == n else np.asarray(gpu_valid).astype(bool)
    m = o.mv_min_clearance(idx, check_env=check_env, stop_below=-margin, threads=THREADS, priority=priority)
    exp = m >= 0
    dec = np.abs(m) > margin
    bad = np.nonzero(dec & (g != exp))[0]
    assert len(bad) == 0, f"MV mismatch on decidable queries {idx[bad][:10]} (oracle min clearance {m[bad][:10]})"
    und = ~dec
    assert np.all(~g[und] | (m[und] > -margin)), "GPU says valid where the oracle collides beyond the margin"
    assert np.all(g[und] | (m[und] < margin)), "GPU says invalid where the oracle is clear beyond the margin"
    return len(idx), int(und.sum())


def _key(c):
    """Lexicographic (t, i, j) order; no conflict sorts after every conflict."""
    return (np.inf, 0, 0) if c[0] < 0 else (int(c[0]), int(c[1]), int(c[2]))


def check_ffc(o, gpu_conf, idx=None, margin=MARGIN):
    """Returns (n_checked, n_undecidable).  Decidable queries: identical
    (t, i, j).  Undecidable ones: the GPU answer may not come after the
    oracle's first pair deeper than -margin (a collision no rounding can
    hide), and a reported pair must be within +margin of colliding."""
    n = o.w.batch.n_queries
    idx = np.arange(n) if idx is None else np.asarray(idx)
    g = np.asarray(gpu_conf).reshape(-1, 3)
    g = g[idx] if len(g) == n else g
    exp = o.ffc(idx, threads=THREADS)
    dec = o.ffc_decidable(idx, margin=margin, threads=THREADS)
    bad = np.nonzero(dec & np.any(g != exp, axis=1))[0]
    assert len(bad) == 0, f"FFC mismatch on decidable queries {idx[bad][:10]}: gpu {g[bad][:5]} oracle {exp[bad][:5]}"
    und = np.nonzero(~dec)[0]
    if len(und):
        deep = o.ffc_below(-margin, idx[und], threads=THREADS)
        for k, d in zip(und, deep):
            q = int(idx[k])
            assert _key(g[k]) <= _key(d), \
                f"query {q}: GPU answer {tuple(g[k])} passes over the deep conflict {tuple(d)}"
            t, i, j = (int(v) for v in g[k])
            if t >= 0:
                nrob = int(o.w.batch.q_robot_off[q + 1] - o.w.batch.q_robot_off[q])
                assert 0 <= i < j < nrob, f"query {q}: bad pair {(i, j)}"
                p = i * nrob - i * (i + 1) // 2 + (j - i - 1)
                c = o.pair_clearances(q, t)[p]
                assert c < margin, f"query {q}: reported pair {(t, i, j)} is clear by {c}"
    return len(idx), int(len(und))


def sample(n, k, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(n, k), replace=False))
