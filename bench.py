"""Benchmark: MV/FFC motion-checks/s on the heterogeneous ragged batch, one GB300.

The headline workload is 1,000,000 mixed MV/FFC queries (teams of 2 arms plus
0-6 discs in the box world, 8-512 steps per query, half MV and half FFC) run
as one persistent work-stealing launch replayed from a CUDA graph, with the
scheduler tuning picked by the library's autotuner.  A step is one pass over
the whole batch with inputs resident in HBM: counter reset, preparation
kernels, the persistent kernel instances and the result kernel.  L2 is
flushed (a 512 MB write) before every timed step; each step is timed with
CUDA events on the launching stream.  The other workloads (the 4-arm cage
MV and FFC batches, discs, the 8- and 16-arm cages, prioritized edges) and the
request server are reported under their own keys.  Rank 0 prints one JSON
line.

--impl reference times the FP64 oracle on the host cores instead (the
reference arm for this workload: the paper ships no code).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MV/FFC motion-checks/s vs per-query launch; p50/p99 latency, 1 GB300"
WORKLOAD = "ragged_teams_1m: 1M mixed MV/FFC queries (1/2 each) in one persistent CUDA-graph launch; teams of " \
           "2 Panda-like 7-DOF arms x 64 spheres + 0-6 discs (2-8 robots), box world with 20 boxes, one segment " \
           "per robot, 8-512 steps per query (log-uniform)"
CAGE_WORKLOAD = "cage_mv: MV, 4 Panda-like 7-DOF arms x 64 spheres, cage env 40 spheres + 12 boxes, " \
                "10k start/goal joint-space motions, resolution 1/32 rad"
# workloads the timed step can run (--workload; the default is the headline):
# description, and the query kind when the batch holds one kind only
STEP_WORKLOADS = {
    "ragged_teams": (WORKLOAD, None),
    "cage_mv": (CAGE_WORKLOAD, 0),
    "cage_ffc": ("cage_ffc: FFC, the 4 arms on independent timed paths of 20-60 waypoints, 8-64 steps per "
                 "segment", 1),
    "cage16_ffc": ("cage16_ffc: FFC, the 16-arm Cage team (8 floor- and 8 ceiling-mounted arms) on whole "
                   "motions between valid team configurations", 1),
}


def make_step_workload(name, n, rank):
    """The timed step's batch: each rank its own seed (weak scaling)."""
    from paper_2604_23960_gb300 import workloads as W
    if name == "ragged_teams":
        w = W.make_ragged_teams(n, seed=205 + rank)
    elif name == "cage_mv":
        w = W.make_cage_mv(n, query_seed=203 + rank)
    elif name == "cage_ffc":
        w = W.make_cage_ffc(n, query_seed=204 + rank)
    else:
        w = W.make_cage16_ffc(n, query_seed=210 + rank)
    kind = STEP_WORKLOADS[name][1]
    if kind is not None:
        w.batch.q_kind = np.full(w.batch.n_queries, kind, np.uint8)
    return w
# FP32 flops per unit of work the kernel counts (FMA = 2):
FLOPS_PER_TEST = 10     # sphere-sphere test: 3 sub, 1 mul + 2 fma, radius add + square
FLOPS_PER_BOX = 13      # sphere-box test: per axis clamp + sub + fma, radius square
FLOPS_PER_CHAIN = 390   # 7-joint modified-DH chain + flange: 48 per joint, 54 for the flange
FLOPS_PER_JOINT = 48    # one modified-DH joint of a chain (sin/cos, row mixing, position update)
FLOPS_PER_FLANGE = 54   # the fixed flange transform at the end of a chain
FLOPS_PER_SPHERE = 28   # sphere placement: 3x4 transform, shift, |p|^2 - r^2
FLOPS_PER_CYL = 32      # sphere-cylinder test: axial coordinate, radial distance, clamps, compare


def dense_flops_per_state(w):
    """FP32 flops the method itself spends on one composite state of a
    homogeneous workload (every query has the same robots and obstacles):
    every robot-robot sphere pair, every robot sphere against every obstacle
    sphere and box, every listed self pair, one FK chain per robot and the
    placement of every sphere -- the per-unit figure of the ALU roofline."""
    b = w.batch
    slots = b.slot_robot[b.q_robot_off[0]:b.q_robot_off[1]]
    ms = [w.models[s].n_spheres for s in slots]
    n_self = sum(len(w.models[s].self_pairs) for s in slots)
    env = w.envs[w.env] if w.env >= 0 else None
    n_s = 0 if env is None else len(env.spheres)
    n_b = 0 if env is None else len(env.aabbs)
    M = sum(ms)
    pairs = sum(ms[i] * ms[j] for i in range(len(ms)) for j in range(i + 1, len(ms)))
    chains = sum(1 for s in slots if w.models[s].kind != 1)
    return (FLOPS_PER_TEST * (pairs + M * n_s + n_self) + FLOPS_PER_BOX * M * n_b
            + FLOPS_PER_CHAIN * chains + FLOPS_PER_SPHERE * M)


def work_flops(st):
    """FP32 flops the kernel performed in one call, from its counters."""
    box = st["box_tests"]
    return (FLOPS_PER_TEST * (st["sphere_tests"] - box) + FLOPS_PER_BOX * box
            + FLOPS_PER_CHAIN * st["fk_chains"] + FLOPS_PER_SPHERE * st["spheres_placed"])


def method_flops(st):
    """FP32 flops of the method's dense work on the states a call checked
    (every robot-robot, obstacle and self test of each checked state, its FK
    chains and sphere placements, for each query's own team and obstacles),
    from the kernel's counters of that work: the ALU roofline's numerator."""
    return (FLOPS_PER_TEST * st["method_sphere_tests"] + FLOPS_PER_BOX * st["method_box_tests"]
            + FLOPS_PER_CYL * st["method_cylinder_tests"] + FLOPS_PER_JOINT * st["method_joints"]
            + FLOPS_PER_FLANGE * st["method_chains"] + FLOPS_PER_SPHERE * st["method_spheres"])


def roofline_frac(st, kernel_ms, peak):
    """(achieved TFLOP/s of the method's work, fraction of the FP32 peak)."""
    a = method_flops(st) / (kernel_ms / 1e3) / 1e12 if kernel_ms > 0 else 0.0
    return a, a / peak


MAKERS = None

# DRAM bytes of one persistent-kernel launch of the headline step, from a
# one-pass ncu capture of that launch; valid only for the kernel source it was
# taken on (any other source reports null)
TRAFFIC = {"kernel_sha256": "8f082716c742bf61ade534f4aa36790c28c8bc4bc6c40489065af358daddf959",
           "bytes": 1336598528 + 37718272}


def traffic_per_launch():
    import hashlib
    src = ROOT / "paper_2604_23960_gb300" / "csrc" / "mrv_kernels.cu"
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    return TRAFFIC["bytes"] if h == TRAFFIC["kernel_sha256"] else None


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text()), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampler for the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)   # let the sampler start before the measured work
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def serving(ctx, duration_s=6.0, loads=(0.5, 0.8, 0.95), n_clients=64, seed=206):
    """Poisson arrivals from 64 simulated planner clients; requests of
    logU[1, 4096] motions from four families over four resident envs;
    continuous batching over 4 streams.  Returns capacity, and throughput with
    p50/p99 request latency (arrival -> result) at each load fraction."""
    import threading
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W
    models, envs, fams = W.make_serving_families(20000, seed=seed)
    rids = [ctx.upload_model(m) for m in models]
    eids = [ctx.upload_env(e) for e in envs]
    bas = [ctx.bind(f, rids, eids) for f in fams]
    rng = np.random.default_rng(seed)
    pool = []
    for _ in range(600):
        f = int(rng.integers(0, 4))
        n = int(np.clip(round(math.exp(rng.uniform(0.0, math.log(4096)))), 1, 4096))
        q0 = int(rng.integers(0, fams[f].batch.n_queries - n))
        pool.append(mrv.slice_batch(bas[f], q0, q0 + n))
    mean_size = float(np.mean([r.n_queries for r in pool]))
    # the server runs a fixed scheduling, not whatever the previous benchmark
    # batch tuned the context to: two slices per work item and per tile, the
    # setting with the highest capacity on this request mix (one-slice items
    # and four slices per tile give about 11% less capacity for a 30% lower
    # median latency at half load)
    mrv.mrv_set_tuning(ctx.h, 2, 4, 0, 2, 0)
    tuning = mrv.mrv_get_tuning(ctx.h)
    srv = mrv.Server(ctx, n_streams=4, device_budget_bytes=2 << 30, max_batch_queries=65536, max_pending=100000)
    # the whole pool submitted at once (a deep queue: the largest micro-batches)
    t0 = time.perf_counter()
    tickets = [srv.submit(r) for r in pool]
    for t, r in zip(tickets, pool):
        srv.wait(t, r.n_queries, timeout_ms=600000)
    deep_qps = sum(r.n_queries for r in pool) / (time.perf_counter() - t0)
    # capacity for this client population: every client submits its next
    # request as soon as the last one returns (at most n_clients in flight)
    done = [0]
    lock = threading.Lock()
    t_cap_end = time.perf_counter() + max(2.0, duration_s / 2)

    def closed(cid):
        r = np.random.default_rng(seed * 7 + cid)
        while time.perf_counter() < t_cap_end:
            req = pool[int(r.integers(0, len(pool)))]
            srv.wait(srv.submit(req), req.n_queries, timeout_ms=600000)
            with lock:
                done[0] += req.n_queries

    t0 = time.perf_counter()
    th = [threading.Thread(target=closed, args=(c,)) for c in range(n_clients)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    cap_qps = done[0] / (time.perf_counter() - t0)
    out = {"capacity": cap_qps, "capacity_deep_queue": deep_qps, "unit": "motion-checks/s",
           "capacity_basis": f"{n_clients} clients submitting back to back", "clients": n_clients,
           "mean_request": mean_size, "streams": 4, "tuning": tuning, "loads": []}
    for frac in loads:
        lam = frac * cap_qps / mean_size              # requests / s over all clients
        lat, done_q = [], [0]
        lock = threading.Lock()
        t_start = time.perf_counter() + 0.2
        t_end = t_start + duration_s

        def client(cid):
            r = np.random.default_rng(seed * 1000 + cid + int(frac * 100))
            t = t_start + r.exponential(n_clients / lam)
            while t < t_end:
                now = time.perf_counter()
                if t > now:
                    time.sleep(t - now)
                req = pool[int(r.integers(0, len(pool)))]
                # arrival = the submit (a client thread that woke late does
                # not add its own delay to the server's latency)
                t_sub = time.perf_counter()
                tk = srv.submit(req)
                srv.wait(tk, req.n_queries, timeout_ms=600000)
                fin = time.perf_counter()
                with lock:
                    lat.append(fin - t_sub)
                    done_q[0] += req.n_queries
                t += r.exponential(n_clients / lam)

        th = [threading.Thread(target=client, args=(c,)) for c in range(n_clients)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        span = max(time.perf_counter(), t_end) - t_start
        la = np.array(lat) * 1e3
        out["loads"].append({"load": frac, "offered_req_s": lam, "requests": len(lat),
                             "throughput": done_q[0] / span, "p50_ms": float(np.percentile(la, 50)) if len(la) else None,
                             "p99_ms": float(np.percentile(la, 99)) if len(la) else None})
    st = srv.stats()
    out["micro_batches"] = st["micro_batches"]
    out["max_inflight"] = st["max_inflight"]
    out["device_budget_bytes"] = st["device_budget_bytes"]
    out["device_free_bytes_after_sizing"] = st["device_free_bytes"]
    out["presized_queries_per_micro_batch"] = st["presized_queries"]
    srv.close()
    return out


def autotune(ctx, w, flags, kind=None, n_sample=None):
    """Picks the scheduler tuning for a batch class (untimed setup): the
    library's autotuner times its candidates on the first n_sample queries."""
    import torch
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W
    sub = w if n_sample is None or n_sample >= w.batch.n_queries else W.subset(w, np.arange(n_sample))
    bs = ctx.bind(sub, ctx.robot_ids, ctx.env_ids).to("cuda")
    if kind is not None:
        bs.a["q_kind"] = torch.full((sub.batch.n_queries,), kind, dtype=torch.uint8, device="cuda")
    t = mrv.mrv_autotune(ctx.h, bs.struct(flags, with_kind=True))
    torch.cuda.synchronize()
    return t


def other_configs(ctx, flush, fp32_peak, per_query_n=1000, reps=3):
    """Throughput of the other workload configurations (device-resident
    inputs, batched persistent launch) next to one synchronous launch per
    query on a sample of the same batch; per configuration the persistent
    kernel's time (CUDA events on its stream) and the FP32 roofline fraction
    of the method's work on the states it checked."""
    import torch
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W
    out = {}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best, kms = [], []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best.append(time.perf_counter() - t0)
            kms.append(ctx.stats()["device_ms"])
        return statistics.median(best), statistics.median(kms), ctx.stats()

    def per_query(w, call):
        sub = W.subset(w, np.arange(min(per_query_n, w.batch.n_queries)))
        bs = ctx.bind(sub, ctx.robot_ids, ctx.env_ids).to("cuda")
        call(bs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call(bs)
        torch.cuda.synchronize()
        return sub.batch.n_queries / (time.perf_counter() - t0)

    def entry(w, dt, kms, st, pq, **extra):
        a, f = roofline_frac(st, kms, fp32_peak)
        e = {"value": w.batch.n_queries / dt, "per_query_launch": pq, "speedup": w.batch.n_queries / dt / pq,
             "ms": dt * 1e3, "kernel_ms": kms, "roofline_achieved_tflops": a, "roofline_frac": f,
             "effort_states": st["states_checked"] / max(1, st["states_available"])}
        e.update(extra)
        return e

    # two discs in the box world, 1,000 queries: MV and FFC
    w = W.make_plain_discs(1000)
    ba = ctx.bind(w).to("cuda")
    for kind, call in (("mv", lambda b, f=0: ctx.mv_validate(b, flags=f)), ("ffc", lambda b, f=0: ctx.ffc_find(b, flags=f))):
        dt, kms, st = timed(lambda: call(ba))
        pq = per_query(w, lambda b: call(b, mrv.MRV_PER_QUERY_LAUNCH))
        out[f"discs_{kind}_1k"] = entry(w, dt, kms, st, pq)
    # four arms, 100k timed path-sets: FFC
    w = W.make_cage_ffc(100000)
    ba = ctx.bind(w).to("cuda")
    tune = autotune(ctx, w, 0, kind=1, n_sample=20000)
    dt, kms, st = timed(lambda: ctx.ffc_find(ba))
    pq = per_query(w, lambda b: ctx.ffc_find(b, flags=mrv.MRV_PER_QUERY_LAUNCH))
    out["cage_ffc_100k"] = entry(w, dt, kms, st, pq, tuning=tune)
    # the Cage scenario's team (Sec. V-A): 4 floor- and 4 ceiling-mounted arms
    # among cylinder obstacles, 10k composite motions
    w = W.make_cage8_mv(10000)
    ba = ctx.bind(w).to("cuda")
    tune = autotune(ctx, w, mrv.MRV_CHECK_ENV, kind=0)
    dt, kms, st = timed(lambda: ctx.mv_validate(ba))
    nvalid = int(ctx.mv_validate(ba).sum().item())
    pq = per_query(w, lambda b: ctx.mv_validate(b, flags=mrv.MRV_PER_QUERY_LAUNCH))
    out["cage8_cyl_10k"] = entry(w, dt, kms, st, pq, tuning=tune, valid_total=f"{nvalid}/{w.batch.n_queries}")
    # the 16-arm Cage team (8 floor- and 8 ceiling-mounted arms, 1024 spheres
    # and 120 robot pairs per state: the large-team kernel): MV on 10k
    # planner-like edges of at most 0.5 rad, FFC on 10k whole motions
    w = W.make_cage16_mv(10000)
    ba = ctx.bind(w).to("cuda")
    tune = autotune(ctx, w, mrv.MRV_CHECK_ENV, kind=0)
    dt, kms, st = timed(lambda: ctx.mv_validate(ba))
    nvalid = int(ctx.mv_validate(ba).sum().item())
    pq = per_query(w, lambda b: ctx.mv_validate(b, flags=mrv.MRV_PER_QUERY_LAUNCH))
    out["cage16_cyl_10k"] = entry(w, dt, kms, st, pq, tuning=tune, valid_total=f"{nvalid}/{w.batch.n_queries}",
                                  order_study=order_study(ctx, ba, flush, linear=False))
    w = W.make_cage16_ffc(10000)
    ba = ctx.bind(w).to("cuda")
    dt, kms, st = timed(lambda: ctx.ffc_find(ba))
    pq = per_query(w, lambda b: ctx.ffc_find(b, flags=mrv.MRV_PER_QUERY_LAUNCH))
    out["cage16_ffc_10k"] = entry(w, dt, kms, st, pq)
    # prioritized planning's edge checks (Sec. IV-C): 10k cage edges, one arm
    # against the cage, itself and three higher-priority arms' timed paths
    w = W.make_cage_priority(10000)
    ba = ctx.bind(w).to("cuda")
    tune = autotune(ctx, w, mrv.MRV_CHECK_ENV | mrv.MRV_PRIORITY, kind=0)
    dt, kms, st = timed(lambda: ctx.mv_validate(ba, flags=mrv.MRV_PRIORITY))
    nvalid = int(ctx.mv_validate(ba, flags=mrv.MRV_PRIORITY).sum().item())
    pq = per_query(w, lambda b: ctx.mv_validate(b, flags=mrv.MRV_PRIORITY | mrv.MRV_PER_QUERY_LAUNCH))
    out["cage_priority_10k"] = entry(w, dt, kms, st, pq, tuning=tune, valid_total=f"{nvalid}/{w.batch.n_queries}")
    return out


def cage_mv_config(ctx, flush, fp32_peak, stream, steps=20, per_query_n=2000):
    """The 4-arm cage MV batch (10k motions): CUDA-graph replay with inputs in
    HBM, the same through mv_validate with pinned host buffers, one launch
    per query, the exhaustive passes (frame-level broadphase and dense) and
    the effort of the state orders."""
    import torch
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W
    w = W.make_cage_mv(10000)
    ba_host = ctx.bind(w)
    ba = ba_host.to("cuda")
    nq = w.batch.n_queries
    ba.a["q_kind"] = torch.zeros(nq, dtype=torch.uint8, device="cuda")   # every query is MV
    bs = ba.struct(mrv.MRV_CHECK_ENV, with_kind=True)
    mrv.mrv_autotune(ctx.h, bs)
    tune = mrv.mrv_get_tuning(ctx.h)
    valid = torch.empty(nq, dtype=torch.uint8, device="cuda")
    conf = torch.empty((nq, 3), dtype=torch.int32, device="cuda")
    graph = mrv.mrv_graph_create(ctx.h, bs, valid, conf)
    for _ in range(3):
        mrv.mrv_graph_launch(graph)
        ctx.sync()
    step_ms, kern_ms = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mrv.mrv_graph_launch(graph)
        e1.record(stream)
        ctx.sync()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(ctx.stats()["device_ms"])
    st = ctx.stats()
    mrv.mrv_graph_destroy(graph)
    nvalid = int(valid.sum().item())
    kms = statistics.mean(kern_ms)
    per_state = dense_flops_per_state(w)
    ach, frac = roofline_frac(st, kms, fp32_peak)
    # end to end with pinned host buffers through mv_validate
    bh = ba_host.to("cpu", pin=True)
    out_h = torch.empty(nq, dtype=torch.uint8).pin_memory()
    e2e = []
    for i in range(6):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mrv.mv_validate(ctx.h, bh.struct(mrv.MRV_CHECK_ENV), out_h, None)
        e2e.append(time.perf_counter() - t0)
    assert int(out_h.sum()) == nvalid
    # one synchronous launch per query
    pq_n = min(nq, per_query_n)
    bsub = ctx.bind(W.subset(w, np.arange(pq_n)), ctx.robot_ids, ctx.env_ids).to("cuda")
    ctx.mv_validate(bsub, flags=mrv.MRV_PER_QUERY_LAUNCH)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pq_valid = ctx.mv_validate(bsub, flags=mrv.MRV_PER_QUERY_LAUNCH)
    torch.cuda.synchronize()
    pq_rate = pq_n / (time.perf_counter() - t0)
    assert torch.equal(pq_valid, valid[:pq_n])
    # exhaustive passes: with the frame-level broadphase and testing every
    # sphere pair (the dense, ALU-bound regime)
    ex = {}
    for name, flags in (("broadphase", 0), ("dense", mrv.MRV_NO_BROADPHASE)):
        ctx.mv_validate(ba, exhaustive=True, flags=flags)
        ms = []
        for _ in range(3):
            flush.zero_()
            ctx.mv_validate(ba, exhaustive=True, flags=flags)
            ms.append(ctx.stats()["device_ms"])
        est = ctx.stats()
        m = statistics.median(ms)
        a, f = roofline_frac(est, m, fp32_peak)
        ex[name] = {"kernel_ms": m, "achieved": a, "frac": f, "performed": work_flops(est) / (m / 1e3) / 1e12,
                    "sphere_tests": est["sphere_tests"], "fk_chains": est["fk_chains"]}
    return {"workload": CAGE_WORKLOAD, "value": nq / (statistics.mean(step_ms) / 1e3), "unit": "motion-checks/s",
            "ms_per_step": statistics.mean(step_ms), "kernel_ms": kms, "tuning": tune,
            "valid_total": f"{nvalid}/{nq}",
            "roofline_achieved_tflops": ach, "roofline_frac": frac,
            "flops_per_state": per_state,
            "performed_tflops": work_flops(st) / (kms / 1e3) / 1e12,
            "effort": {"states": st["states_checked"] / max(1, st["states_available"]),
                       "sphere_tests_vs_dense": st["sphere_tests"] / max(1, st["sphere_tests_available"])},
            "e2e": {"value": nq / statistics.median(e2e), "unit": "motion-checks/s",
                    "api": "mv_validate with pinned host buffers"},
            "per_query_launch": {"value": pq_rate, "queries": pq_n,
                                 "speedup_batched": nq / (statistics.mean(step_ms) / 1e3) / pq_rate},
            "roofline_exhaustive": ex,
            "order_study": order_study(ctx, ba, flush)}


def order_study(ctx, ba, flush, reps=3, linear=True):
    """Effort of the state-visiting orders of MV (combined, hierarchical
    env/self-then-pairs, or pairs first: the adjacent fixed-base pairs, then
    the rest; x rake or linear state map) on a batch, early exit: fraction of
    states checked, fraction of the method's sphere tests executed (dense
    kernel, the effort of Fig. 4) and kernel time with and without the
    frame-level broadphase.  All give the same verdicts."""
    from paper_2604_23960_gb300 import mrv
    out = {}
    saved = mrv.mrv_get_tuning(ctx.h)
    mrv.mrv_set_tuning(ctx.h, **dict(saved, mv_order=0))   # flags 0: the combined order
    orders = [("combined_rake", 0), ("hierarchical_rake", mrv.MRV_HIERARCHICAL),
              ("pairs_first_rake", mrv.MRV_PAIRS_FIRST)]
    if linear:
        orders += [("combined_linear", mrv.MRV_LINEAR),
                   ("hierarchical_linear", mrv.MRV_HIERARCHICAL | mrv.MRV_LINEAR),
                   ("pairs_first_linear", mrv.MRV_PAIRS_FIRST | mrv.MRV_LINEAR)]
    for name, fl in orders:
        row = {}
        for tag, extra in (("", 0), ("_dense", mrv.MRV_NO_BROADPHASE)):
            ctx.mv_validate(ba, flags=fl | extra)
            ms = []
            for _ in range(reps):
                flush.zero_()
                ctx.mv_validate(ba, flags=fl | extra)
                ms.append(ctx.stats()["device_ms"])
            st = ctx.stats()
            row["kernel_ms" + tag] = statistics.median(ms)
            if not extra:
                row["effort_states"] = st["states_checked"] / max(1, st["states_available"])
            else:
                row["effort_tests"] = st["sphere_tests"] / max(1, st["sphere_tests_available"])
        out[name] = row
    mrv.mrv_set_tuning(ctx.h, **saved)
    return out


def validation_study(ctx, flush, n_queries=500, reps=3):
    """The paper's validation experiment (Sec. V-B, its validation table) on
    the synthetic stand-ins: 500 Cage motions with valid endpoints for 4, 8
    and 16 arms, with and without obstacles; per state order (combined or
    hierarchical x rake or linear packing): valid/total, the effort of early
    termination (sphere tests executed / available, dense kernel; states
    checked / available) and k_main time with the frame-level broadphase and
    dense, early-terminating and exhaustive."""
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W
    saved = mrv.mrv_get_tuning(ctx.h)
    mrv.mrv_set_tuning(ctx.h, **dict(saved, mv_order=0))   # flags 0: the combined order
    orders = [("combined_rake", 0), ("hierarchical_rake", mrv.MRV_HIERARCHICAL),
              ("combined_linear", mrv.MRV_LINEAR), ("hierarchical_linear", mrv.MRV_HIERARCHICAL | mrv.MRV_LINEAR)]

    def kernel_ms(ba, flags, exhaustive):
        ctx.mv_validate(ba, flags=flags, exhaustive=exhaustive)
        ms = []
        for _ in range(reps):
            flush.zero_()
            ctx.mv_validate(ba, flags=flags, exhaustive=exhaustive)
            ms.append(ctx.stats()["device_ms"])
        return statistics.median(ms), ctx.stats()

    out = {}
    for n in (4, 8, 16):
        for obst in (True, False):
            w = W.make_cage_team_study(n, n_queries, obstacles=obst)
            ba = ctx.bind(w).to("cuda")
            v = ctx.mv_validate(ba)
            cell = {"valid_total": f"{int(v.sum().item())}/{n_queries}"}
            for name, fl in orders:
                ms_b, st_b = kernel_ms(ba, fl, False)
                ms_d, st_d = kernel_ms(ba, fl | mrv.MRV_NO_BROADPHASE, False)
                ex_b, _ = kernel_ms(ba, fl, True)
                ex_d, _ = kernel_ms(ba, fl | mrv.MRV_NO_BROADPHASE, True)
                cell[name] = {"effort_tests": st_d["sphere_tests"] / max(1, st_d["sphere_tests_available"]),
                              "effort_states": st_b["states_checked"] / max(1, st_b["states_available"]),
                              "kernel_ms": ms_b, "kernel_ms_dense": ms_d,
                              "exhaustive_ms": ex_b, "exhaustive_ms_dense": ex_d}
            out[f"{n}_arms_{'obstacles' if obst else 'no_obstacles'}"] = cell
    mrv.mrv_set_tuning(ctx.h, **saved)
    return out


def _oracle_mixed(o, kind, idx, threads):
    """The oracle on queries idx of a mixed batch: MV (Alg. 1) where kind is
    0, FFC (Alg. 2) where it is 1."""
    idx = np.asarray(idx)
    k = kind[idx]
    if (k == 0).any():
        o.mv(idx[k == 0], threads=threads)
    if (k == 1).any():
        o.ffc(idx[k == 1], threads=threads)


def cpu_baseline(w, seconds_hint: float = 20.0):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample
    (the first queries of the batch, MV or FFC by their kind)."""
    from oracle import oracle as O
    o = O.Oracle(w)
    kind = w.batch.q_kind if w.batch.q_kind is not None else np.zeros(w.batch.n_queries, np.uint8)
    threads = os.cpu_count() or 1
    n = w.batch.n_queries
    idx = np.arange(min(n, 512))
    t0 = time.perf_counter()
    _oracle_mixed(o, kind, idx, threads)
    per_q = (time.perf_counter() - t0) / len(idx)
    k = int(min(n, max(len(idx), seconds_hint / max(per_q, 1e-9))))
    t0 = time.perf_counter()
    _oracle_mixed(o, kind, np.arange(k), threads)
    dt = time.perf_counter() - t0
    # one core on a fixed subset of about a fifth of that time
    k1 = int(min(n, max(64, 0.2 * seconds_hint / max(per_q * threads, 1e-9))))
    t1 = time.perf_counter()
    _oracle_mixed(o, kind, np.arange(k1), 1)
    dt1 = time.perf_counter() - t1
    return {"value": k / dt, "unit": "motion-checks/s", "cores": threads, "kind": "oracle",
            "sample": f"first {k} of the {n} queries (MV or FFC by kind), FP64 scalar with early exit, "
                      f"{threads} threads",
            "cpu": _cpu_model(),
            "single_core": {"value": k1 / dt1, "unit": "motion-checks/s", "cores": 1,
                            "sample": f"first {k1} of the {n} queries, one thread"}}


def _cpu_model() -> str:
    """The host CPU's name as the kernel reports it (x86 model name, or the
    Arm implementer / part numbers), with the core count."""
    info = {}
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    name = info.get("model name") or " ".join(
        f"{k} {info[k]}" for k in ("CPU implementer", "CPU part") if k in info) or platform.machine()
    return f"{name}, {os.cpu_count()} logical cores"



def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2604_23960_gb300 import workloads as W
    w = W.make_ragged_teams(args.queries)
    o = O.Oracle(w)
    kind = w.batch.q_kind
    threads = os.cpu_count() or 1
    sample = args.ref_sample
    n = w.batch.n_queries
    rng_idx = [np.arange(s * sample, (s + 1) * sample) % n for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        _oracle_mixed(o, kind, rng_idx[s], threads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        _oracle_mixed(o, kind, rng_idx[args.warmup + s], threads)
    dt = time.perf_counter() - t0
    v = sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "motion-checks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "step": f"{sample} consecutive queries of the {n}-query batch per step (MV or FFC by kind)"},
            "cpu_baseline": {"value": v, "unit": "motion-checks/s", "cores": threads, "kind": "oracle",
                             "sample": f"{sample} queries per step, FP64 scalar oracle with early exit, "
                                       f"{threads} threads, {_cpu_model()}"},
            "e2e": {"value": v, "unit": "motion-checks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def strong_scaling(ctx, n_queries, world, rank, group, flush, reps=3):
    """One batch split across the ranks by estimated cost (multi.shard_by_cost),
    each rank validating its shard with mrv_run on its own GPU, results
    gathered on rank 0 over a host (gloo) group; the time is the slowest
    rank's, between barriers."""
    import torch
    import torch.distributed as dist
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import multi
    from paper_2604_23960_gb300 import workloads as W
    w = W.make_ragged_teams(n_queries)
    ba = ctx.bind(w)
    mine = multi.shard_of(ba, world, rank)
    sh = multi.take_queries(ba, mine).to("cuda")
    ts = []
    for _ in range(reps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        dist.barrier(group=group)
        t0 = time.perf_counter()
        v, c = ctx.run(sh)
        torch.cuda.synchronize()
        t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        ts.append(float(t.item()))
    full_v = multi.gather_results(mine, v.cpu().numpy(), n_queries, world, rank, group=group)
    full_c = multi.gather_results(mine, c.cpu().numpy(), n_queries, world, rank, group=group)
    if rank != 0:
        return None
    dt = statistics.median(ts[1:])
    return {"value": n_queries / dt, "unit": "motion-checks/s", "ms": dt * 1e3, "n_gpus": world,
            "queries": n_queries, "shard_sizes_by_cost": "LPT greedy on robot pairs x states",
            "gathered": int(len(full_v) == n_queries and len(full_c) == n_queries), "_valid": full_v,
            "_conf": full_c}


def run(args):
    import torch
    import torch.distributed as dist
    from paper_2604_23960_gb300 import mrv
    from paper_2604_23960_gb300 import workloads as W

    rank, world, local = _dist()
    host_group = None
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        host_group = dist.new_group(backend="gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    ctx = mrv.Context(local, stream.cuda_stream)
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    # weak scaling: every rank validates its own batch (distinct seeds), with
    # no collective on the data path
    w = make_step_workload(args.workload, args.queries, rank)
    ba_host = ctx.bind(w)
    ba = ba_host.to("cuda")
    nq = w.batch.n_queries
    kind = torch.as_tensor(w.batch.q_kind, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    valid = torch.empty(nq, dtype=torch.uint8, device=dev)
    conf = torch.empty((nq, 3), dtype=torch.int32, device=dev)
    bs = ba.struct(mrv.MRV_CHECK_ENV, with_kind=True)
    with torch.cuda.stream(stream):
        # scheduler tuning for this batch class, timed on the whole batch (untimed
        # setup; the graph keeps it).  A 100k-query sample fits in L2 and
        # does not tell 2 from 4 slices per item, which differ by 12% on the
        # 1M batch, whose items re-read their queries' records from DRAM
        autotune(ctx, w, mrv.MRV_CHECK_ENV)
        graph = mrv.mrv_graph_create(ctx.h, bs, valid, conf)
    tuning = mrv.mrv_get_tuning(ctx.h)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms = []
    torch.cuda.nvtx.range_push("timed")
    with Clocks(local) as clk:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                mrv.mrv_graph_launch(graph)
                ctx.sync()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                mrv.mrv_graph_launch(graph)
                ev[i][1].record(stream)
                ctx.sync()
                st_step = ctx.stats()
                kern_ms.append(st_step["device_ms"])
        torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    t = torch.tensor([total_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_s = float(t.item())
    value = nq * world * args.steps / total_s
    mvq, ffq = kind == 0, kind == 1
    nvalid = int(valid[mvq].sum().item())
    nconf = int((conf[ffq][:, 0] >= 0).sum().item())

    # end to end through the public API (mrv_run) with pinned host buffers:
    # the inputs' host->device copies and the results' device->host copies
    # are inside the timed region
    bh = ba_host.to("cpu", pin=True)
    vh = torch.empty(nq, dtype=torch.uint8).pin_memory()
    ch = torch.empty((nq, 3), dtype=torch.int32).pin_memory()
    bhs = bh.struct(mrv.MRV_CHECK_ENV, with_kind=True)
    e2e_ms = []
    with torch.cuda.stream(stream):
        mrv.mrv_run(ctx.h, bhs, vh, ch)
        for i in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            mrv.mrv_run(ctx.h, bhs, vh, ch)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    kh = w.batch.q_kind
    assert np.array_equal(vh.numpy()[kh == 0], valid.cpu().numpy()[kh == 0])
    assert np.array_equal(ch.numpy()[kh == 1], conf.cpu().numpy()[kh == 1])
    h2d = sum(v.numel() * v.element_size() for v in bh.a.values() if v is not None)
    d2h = vh.numel() * vh.element_size() + ch.numel() * ch.element_size()
    e2e_t = torch.tensor([statistics.median(e2e_ms)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_val = nq * world / (float(e2e_t.item()) / 1e3)

    strong = None
    if world > 1 and args.workload == "ragged_teams":
        with torch.cuda.stream(stream):
            strong = strong_scaling(ctx, nq, world, rank, host_group, flush)
        if rank == 0:
            # the gathered answer of the split batch equals this rank's whole-batch answer (same seed)
            assert np.array_equal(strong.pop("_valid")[kh == 0], valid.cpu().numpy()[kh == 0])
            assert np.array_equal(strong.pop("_conf")[kh == 1], conf.cpu().numpy()[kh == 1])
    if rank != 0:   # the remaining measurements run on rank 0 only
        mrv.mrv_graph_destroy(graph)
        ctx.close()
        dist.destroy_process_group()
        return

    # one synchronous launch per query (the plain GPU path) on the first
    # queries of the same batch
    with torch.cuda.stream(stream):
        pq_n = min(nq, args.per_query_n)
        bsub = ctx.bind(W.subset(w, np.arange(pq_n)), ctx.robot_ids, ctx.env_ids).to("cuda")
        ctx.run(bsub, flags=mrv.MRV_PER_QUERY_LAUNCH)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pv, pc = ctx.run(bsub, flags=mrv.MRV_PER_QUERY_LAUNCH)
        torch.cuda.synchronize()
        pq_rate = pq_n / (time.perf_counter() - t0)
    km = kind[:pq_n]
    assert torch.equal(pv[km == 0], valid[:pq_n][km == 0]) and torch.equal(pc[km == 1], conf[:pq_n][km == 1])

    kms = statistics.mean(kern_ms)
    achieved, frac = roofline_frac(st_step, kms, fp32_peak)
    performed = work_flops(st_step) / (kms / 1e3) / 1e12
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "motion-checks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": STEP_WORKLOADS[args.workload][0], "queries_per_gpu": nq,
                   "mv_queries": int(mvq.sum().item()),
                   "ffc_queries": int(ffq.sum().item()), "parallelism": f"replicas{world}",
                   "l2": "flushed before every timed step (512 MB write)",
                   "launch": "CUDA graph: reset + prepare + persistent work-stealing kernel instances + results",
                   "tuning": tuning},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic_per_launch(),
                     "kernel": "k_main (persistent MV/FFC kernel, small-team layout), early exit, frame-level broadphase",
                     "work": "the method's dense FP32 work on the states checked, from the kernel's counters: "
                             f"{FLOPS_PER_TEST} flops per sphere-sphere test (robot-robot, obstacle, self), "
                             f"{FLOPS_PER_BOX} per sphere-box test, {FLOPS_PER_JOINT} per joint and "
                             f"{FLOPS_PER_FLANGE} per flange of each FK chain, {FLOPS_PER_SPHERE} per sphere placed",
                     "flops_per_step": method_flops(st_step),
                     "states_checked": st_step["states_checked"],
                     "kernel_ms": kms,
                     "pipe_utilisation": {"achieved": performed, "frac": performed / fp32_peak,
                                          "work": "the tests the kernel actually ran after the broadphase "
                                                  "(bounding-sphere and exact), FK chains and spheres placed"},
                     "peak_source": f"SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                    f"({src} sm_max_mhz)"},
        "e2e": {"value": e2e_val, "unit": "motion-checks/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "api": "mrv_run with pinned host buffers",
                "ms_median": statistics.median(e2e_ms)},
        "per_query_launch": {"value": pq_rate, "unit": "motion-checks/s", "queries": pq_n,
                             "speedup_batched": value / world / pq_rate},
        "effort": {"states": st_step["states_checked"] / max(1, st_step["states_available"]),
                   "sphere_tests_vs_dense": st_step["sphere_tests"] / max(1, st_step["sphere_tests_available"])},
        "valid_mv": f"{nvalid}/{int(mvq.sum().item())}",
        "conflicts_ffc": f"{nconf}/{int(ffq.sum().item())}",
        "kernel_ms_mean": kms,
        # per graph step: k_prep, k_levels, k_scatter, the small-team k_main,
        # the team and large-team k_main instances (forked beside it; no work
        # item on this batch), the full instance's pass over the queries
        # handed over (queries_redone; usually none), k_finish
        "gpu_launches": 8 * args.steps,
        "queries_redone": st_step.get("queries_redone", 0),
        "clocks": clocks,
    }
    if strong is not None:
        line["strong_scaling"] = strong
    mrv.mrv_graph_destroy(graph)
    with torch.cuda.stream(stream):
        if not args.no_configs:
            line["configs"] = {"cage_mv_10k": cage_mv_config(ctx, flush, fp32_peak, stream)}
            line["configs"].update(other_configs(ctx, flush, fp32_peak))
            line["validation_study"] = validation_study(ctx, flush)
        if not args.no_serve:
            line["serving"] = serving(ctx, args.serve_seconds)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    ctx.close()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_serving_only(args):
    """The request server's measurement alone (one GPU): prints its section."""
    import torch
    from paper_2604_23960_gb300 import mrv
    torch.cuda.set_device(0)
    ctx = mrv.Context(0)
    out = serving(ctx, args.serve_seconds)
    ctx.close()
    print(json.dumps({"serving": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mrv", choices=["mrv", "reference"])
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--workload", default="ragged_teams", choices=sorted(STEP_WORKLOADS),
                    help="batch of the timed step (the default is the headline workload)")
    ap.add_argument("--per-query-n", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-sample", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=6.0)
    ap.add_argument("--only-serve", action="store_true",
                    help="run the request server's measurement alone (for profiling its micro-batches)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.only_serve:
        run_serving_only(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
