"""Inputs and calls shared by the bounds-checked build's test.

results(ctx) runs a fixed set of seeded inputs through every path of the
library (MV in each order, flag and layout, FFC, mixed runs, graph replay,
exhaustive minimum clearance, the per-sphere clearance diagnostic, one
launch per query, prioritized MV, cylinders, the large-team kernel instance,
and benchmark-sized batches of the ragged teams, timed-path FFC, 8- and
16-arm workloads) and returns the outputs by name.  The test runs it once in a child process
that loads libmrv_checked.so (MRV_LIBRARY=checked) and once in its own
process with libmrv.so, and compares.  Run as a script, it writes the
outputs to an .npz file; any index check failing in the checked build
surfaces as an MrvError (MRV_ERR_CUDA), so the script exits non-zero.
"""
from __future__ import annotations

import sys

import numpy as np


def _np(x):
    return x if isinstance(x, np.ndarray) else x.cpu().numpy()


def results(ctx) -> dict:
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W
    from tests.tiny import tiny_workload
    out = {}
    orders = {"comb": 0, "hier": mrv.MRV_HIERARCHICAL, "lin": mrv.MRV_LINEAR, "pf": mrv.MRV_PAIRS_FIRST,
              "dense": mrv.MRV_NO_BROADPHASE, "pfdense": mrv.MRV_PAIRS_FIRST | mrv.MRV_NO_BROADPHASE}
    # tiny random teams: point robots and short chains, 1-8 robots, both motion forms
    for seed in range(4):
        for timed in (True, False):
            w = tiny_workload(3000 + seed, n_queries=40, timed=timed, max_steps=40, max_robots=4 + 4 * (seed & 1),
                              n_models=6)
            ba = ctx.bind(w)
            tag = f"tiny{seed}{int(timed)}"
            for name, fl in orders.items():
                for ce in (True, False):
                    out[f"{tag}_mv_{name}_{int(ce)}"] = _np(ctx.mv_validate(ba, check_env=ce, flags=fl))
            out[f"{tag}_mv_ex"], out[f"{tag}_mc"] = (_np(x) for x in
                                                   ctx.mv_validate(ba, exhaustive=True, min_clearance=True))
            out[f"{tag}_ffc"] = _np(ctx.ffc_find(ba))
            out[f"{tag}_ffc_dense"] = _np(ctx.ffc_find(ba, flags=mrv.MRV_NO_BROADPHASE))
            out[f"{tag}_ffc_ex"] = _np(ctx.ffc_find(ba, exhaustive=True))
            out[f"{tag}_pq"] = _np(ctx.mv_validate(ba, flags=mrv.MRV_PER_QUERY_LAUNCH))
            bd = ba.to("cuda")
            out[f"{tag}_mv_dev"] = _np(ctx.mv_validate(bd))
            out[f"{tag}_prio"] = _np(ctx.mv_validate(ba, flags=mrv.MRV_PRIORITY))
            M = sum(w.models[w.batch.slot_robot[s]].n_spheres for s in range(w.batch.q_robot_off[0],
                                                                             w.batch.q_robot_off[1]))
            out[f"{tag}_clr"] = ctx.clearance(ba, 0, [0], M)
    # edge cases: one robot, no motion, eight arms (512 spheres, the team layout's limit)
    env = W.world_boxes(3)
    d = W.disc_robot(0.25)
    bb = W.BatchBuilder(2, False)
    bb.add([0], [np.array([[0.1, 0.1], [9.9, 9.9]])], None, 0, 0)
    bb.add([0, 0], [np.array([[1.0, 1.0], [1.0, 1.0]]), np.array([[1.2, 1.0], [1.2, 1.0]])], None, 0, -1)
    w = W.Workload("edge", [d], [env], bb.build(0.1), 0, True)
    ba = ctx.bind(w)
    out["edge_mv"], out["edge_ffc"] = _np(ctx.mv_validate(ba)), _np(ctx.ffc_find(ba))
    fx = W.load_cage_fixtures()
    arms = [W.panda_like(W._pose(1.3 * np.cos(a), 1.3 * np.sin(a), 0.0, a + np.pi), fx["self_pairs"])
            for a in np.linspace(0, 2 * np.pi, 8, endpoint=False)]
    rng = np.random.default_rng(5)
    bb = W.BatchBuilder(7, True)
    for _ in range(6):
        paths = [rng.uniform(W.PANDA_LO, W.PANDA_HI, (3, 7)) for _ in arms]
        bb.add(list(range(8)), paths, [rng.integers(10, 40, 2) for _ in arms], 0, -1)
    ba = ctx.bind(W.Workload("eight", arms, [], bb.build(), -1, True))
    out["eight_mv"], out["eight_ffc"] = _np(ctx.mv_validate(ba)), _np(ctx.ffc_find(ba))
    # cage workloads: boxes and spheres, cylinders (8 arms), prioritized edges,
    # the 16-arm team on the large-team instance, timed FFC paths
    for name, w, fl in (("cage", W.make_cage_mv(96), 0), ("cage8", W.make_cage8_mv(96), 0),
                        ("prio", W.make_cage_priority(96), mrv.MRV_PRIORITY), ("c16", W.make_cage16_mv(48), 0)):
        ba = ctx.bind(w).to("cuda")
        for oname in ("comb", "hier", "lin", "pf", "dense"):
            if fl and oname == "pf":
                continue
            out[f"{name}_mv_{oname}"] = _np(ctx.mv_validate(ba, flags=fl | orders[oname]))
        out[f"{name}_mv_ex"], out[f"{name}_mc"] = (_np(x) for x in
                                                 ctx.mv_validate(ba, exhaustive=True, min_clearance=True, flags=fl))
    for name, w in (("cffc", W.make_cage_ffc(48)), ("c16ffc", W.make_cage16_ffc(24))):
        ba = ctx.bind(w).to("cuda")
        out[f"{name}"] = _np(ctx.ffc_find(ba))
        out[f"{name}_dense"] = _np(ctx.ffc_find(ba, flags=mrv.MRV_NO_BROADPHASE))
    # mixed ragged teams through mrv_run and a graph replay
    w = W.make_ragged_teams(1500, seed=906)
    ba = ctx.bind(w).to("cuda")
    v, c = ctx.run(ba)
    out["ragged_v"], out["ragged_c"] = _np(v), _np(c)
    import torch
    vg = torch.zeros_like(v)
    cg = torch.zeros_like(c)
    g = mrv.mrv_graph_create(ctx.h, ba.struct(mrv.MRV_CHECK_ENV, with_kind=True), vg, cg)
    mrv.mrv_graph_launch(g)
    ctx.sync()
    mrv.mrv_graph_destroy(g)
    out["ragged_gv"], out["ragged_gc"] = _np(vg), _np(cg)
    out["ragged_kind"] = np.asarray(w.batch.q_kind)
    # benchmark-sized launches (the configurations bench.py times, smaller
    # counts): ragged teams, timed-path FFC, the 16-arm team
    wb = W.make_ragged_teams(60000, seed=907)
    bb = ctx.bind(wb).to("cuda")
    v, c = ctx.run(bb)
    out["big_ragged_v"], out["big_ragged_c"] = _np(v), _np(c)
    out["big_ragged_kind"] = np.asarray(wb.batch.q_kind)
    out["big_ffc"] = _np(ctx.ffc_find(ctx.bind(W.make_cage_ffc(5000, query_seed=908)).to("cuda")))
    out["big_c16"] = _np(ctx.mv_validate(ctx.bind(W.make_cage16_mv(2000, query_seed=909)).to("cuda")))
    out["big_c8"] = _np(ctx.mv_validate(ctx.bind(W.make_cage8_mv(2000, query_seed=910)).to("cuda")))
    return out


def main(path):
    import torch
    from paper_2604_23960_gb300 import mrv
    torch.cuda.set_device(0)
    ctx = mrv.Context(0)
    res = results(ctx)
    ctx.close()
    np.savez(path, library=str(mrv.LIB_PATH.name), **res)


if __name__ == "__main__":
    main(sys.argv[1])
