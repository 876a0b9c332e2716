"""Python binding of the C ABI in ``include/mrv.h`` (ctypes; marshalling only).

Every computation runs in ``libmrv.so`` (CUDA kernels for sm_103a); this
module only converts arrays to pointers.  Loading fails loudly when the
library has not been built: there is no fallback path.

The raw entry points keep the ABI's names (``robot_model_upload``,
``env_upload``, ``mv_validate``, ``ffc_find``, ``mrv_run``, ``mrv_clearance``,
...).  ``Context`` and ``BatchArrays`` are conveniences that keep the arrays
alive, map workload model / env indices to uploaded ids and choose host or
device pointers (torch CUDA tensors for device-resident batches).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from pathlib import Path
from typing import Optional

import numpy as np

from . import workloads as W

# MRV_LIBRARY=checked loads the bounds-checked build of the same library
# (libmrv_checked.so: every kernel index checked against its array, a failure
# reported as MRV_ERR_CUDA naming the check); unset loads libmrv.so
_LIBRARIES = {"": "libmrv.so", "checked": "libmrv_checked.so"}
if os.environ.get("MRV_LIBRARY", "") not in _LIBRARIES:
    raise ImportError(f"MRV_LIBRARY={os.environ['MRV_LIBRARY']!r}: expected one of {sorted(_LIBRARIES)}")
LIB_PATH = Path(__file__).resolve().parent / _LIBRARIES[os.environ.get("MRV_LIBRARY", "")]

MRV_OK = 0
MRV_CHECK_ENV = 0x1
MRV_HIERARCHICAL = 0x2
MRV_EXHAUSTIVE = 0x4
MRV_PTRS_ON_DEVICE = 0x8
MRV_ASYNC = 0x10
MRV_PER_QUERY_LAUNCH = 0x20
MRV_NO_BROADPHASE = 0x40
MRV_LINEAR = 0x80
MRV_PRIORITY = 0x100
MRV_PAIRS_FIRST = 0x200
MRV_KIND_MV = 0
MRV_KIND_FFC = 1
MRV_MAX_ROBOTS = 16
MRV_MAX_QUERY_SPHERES = 1024
MRV_MAX_STEPS = (1 << 24) - 1
MRV_NOALLOC_MAX_QUERIES = 4096
MRV_NOALLOC_MAX_WAYPOINTS = 65536
ERR_NAMES = {-1: "MRV_ERR_ARG", -2: "MRV_ERR_OOM", -3: "MRV_ERR_NOT_FOUND", -4: "MRV_ERR_CUDA",
             -5: "MRV_ERR_TIMEOUT", -6: "MRV_ERR_BUSY", -7: "MRV_ERR_LIMIT"}

P = C.c_void_p


class RobotDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dof", C.c_int32), ("dh", P), ("flange", P), ("base", P),
                ("point_z", C.c_float), ("n_spheres", C.c_int32), ("sphere_link", P), ("sphere_xyzr", P),
                ("n_self_pairs", C.c_int32), ("self_pairs", P)]


class EnvDesc(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres_xyzr", P), ("n_aabbs", C.c_int32), ("aabb_lohi", P),
                ("n_cylinders", C.c_int32), ("cylinders", P)]


class BatchS(C.Structure):
    _fields_ = [("n_queries", C.c_int32), ("n_slots", C.c_int32), ("n_waypoints", C.c_int32),
                ("env_id", C.c_int32), ("q_robot_off", P), ("slot_robot_id", P), ("slot_wp_off", P),
                ("waypoints", P), ("wp_stride", C.c_int32), ("seg_steps", P), ("resolution", C.c_float),
                ("q_env_id", P), ("q_kind", P), ("flags", C.c_uint32)]


class Conflict(C.Structure):
    _fields_ = [("t", C.c_int32), ("i", C.c_int32), ("j", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("states_available", C.c_uint64), ("states_checked", C.c_uint64), ("sphere_tests", C.c_uint64),
                ("sphere_tests_available", C.c_uint64), ("work_items", C.c_uint64), ("n_valid", C.c_int32),
                ("n_conflicts", C.c_int32), ("device_ms", C.c_float), ("box_tests", C.c_uint64),
                ("fk_chains", C.c_uint64), ("spheres_placed", C.c_uint64), ("cylinder_tests", C.c_uint64),
                ("method_sphere_tests", C.c_uint64), ("method_box_tests", C.c_uint64),
                ("method_cylinder_tests", C.c_uint64), ("method_joints", C.c_uint64),
                ("method_chains", C.c_uint64), ("method_spheres", C.c_uint64), ("queries_redone", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("slices_per_item", C.c_int32), ("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("tile_split", C.c_int32), ("mv_order", C.c_int32)]


class Limits(C.Structure):
    _fields_ = [("kernel_budget_ms", C.c_double)]


class ServerOpts(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("device_budget_bytes", C.c_size_t), ("max_batch_queries", C.c_int32),
                ("max_pending", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("micro_batches", C.c_uint64), ("queries", C.c_uint64), ("max_inflight", C.c_uint64),
                ("busy_ms", C.c_double), ("device_budget_bytes", C.c_uint64), ("device_free_bytes", C.c_uint64),
                ("presized_queries", C.c_uint64)]


# name -> (restype, argtypes)
SIGNATURES = {
    "mrv_create": (C.c_int, [C.POINTER(P), C.c_int, P]),
    "mrv_destroy": (C.c_int, [P]),
    "mrv_last_error": (C.c_char_p, [P]),
    "mrv_set_stream": (C.c_int, [P, P]),
    "robot_model_upload": (C.c_int, [P, C.POINTER(RobotDesc), C.POINTER(C.c_int32)]),
    "env_upload": (C.c_int, [P, C.POINTER(EnvDesc), C.POINTER(C.c_int32)]),
    "mrv_release": (C.c_int, [P, C.c_int32]),
    "mv_validate": (C.c_int, [P, C.POINTER(BatchS), P, P]),
    "ffc_find": (C.c_int, [P, C.POINTER(BatchS), P]),
    "mrv_run": (C.c_int, [P, C.POINTER(BatchS), P, P]),
    "mrv_clearance": (C.c_int, [P, C.POINTER(BatchS), C.c_int32, P, C.c_int32, P]),
    "mv_validate_noalloc": (C.c_int, [P, C.POINTER(BatchS), P]),
    "mrv_sync": (C.c_int, [P]),
    "mrv_set_limits": (C.c_int, [P, C.POINTER(Limits)]),
    "mrv_get_stats": (C.c_int, [P, C.POINTER(Stats)]),
    "mrv_set_tuning": (C.c_int, [P, C.POINTER(Tuning)]),
    "mrv_get_tuning": (C.c_int, [P, C.POINTER(Tuning)]),
    "mrv_autotune": (C.c_int, [P, C.POINTER(BatchS), C.c_char_p, C.POINTER(Tuning)]),
    "mrv_graph_create": (C.c_int, [P, C.POINTER(BatchS), P, P, C.POINTER(P)]),
    "mrv_graph_launch": (C.c_int, [P]),
    "mrv_graph_destroy": (C.c_int, [P]),
    "mrv_server_create": (C.c_int, [P, C.POINTER(ServerOpts), C.POINTER(P)]),
    "mrv_server_destroy": (C.c_int, [P]),
    "mrv_server_submit": (C.c_int, [P, C.POINTER(BatchS), C.POINTER(C.c_uint64)]),
    "mrv_server_wait": (C.c_int, [P, C.c_uint64, C.c_int32, P, P]),
    "mrv_server_get_stats": (C.c_int, [P, C.POINTER(ServerStats)]),
}

_lib = None
_lock = threading.Lock()


class MrvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib() -> C.CDLL:
    """Loads libmrv.so; raises when the CUDA extension has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not LIB_PATH.exists():
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(str(LIB_PATH))
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != MRV_OK:
        msg = lib().mrv_last_error(ctx).decode(errors="replace")
        raise MrvError(rc, msg)


def _ptr(a) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------------------
# raw entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def mrv_create(device: int = 0, stream: Optional[int] = None):
    h = P()
    _check(lib().mrv_create(C.byref(h), device, stream))
    return h


def mrv_destroy(ctx):
    _check(lib().mrv_destroy(ctx))


def mrv_set_stream(ctx, stream):
    _check(lib().mrv_set_stream(ctx, stream), ctx)


def robot_model_upload(ctx, desc: RobotDesc) -> int:
    rid = C.c_int32()
    _check(lib().robot_model_upload(ctx, C.byref(desc), C.byref(rid)), ctx)
    return rid.value


def env_upload(ctx, desc: EnvDesc) -> int:
    eid = C.c_int32()
    _check(lib().env_upload(ctx, C.byref(desc), C.byref(eid)), ctx)
    return eid.value


def mrv_release(ctx, rid: int):
    _check(lib().mrv_release(ctx, rid), ctx)


def mv_validate(ctx, batch: BatchS, valid_out, min_clearance_out=None):
    _check(lib().mv_validate(ctx, C.byref(batch), _ptr(valid_out), _ptr(min_clearance_out)), ctx)


def mv_validate_noalloc(ctx, batch: BatchS, valid_out):
    """MV of a device-resident batch with no allocation during the call (the
    scratch is a static device array; see include/mrv.h for the limits)."""
    _check(lib().mv_validate_noalloc(ctx, C.byref(batch), _ptr(valid_out)), ctx)


def ffc_find(ctx, batch: BatchS, out):
    _check(lib().ffc_find(ctx, C.byref(batch), _ptr(out)), ctx)


def mrv_run(ctx, batch: BatchS, valid_out, conflict_out):
    _check(lib().mrv_run(ctx, C.byref(batch), _ptr(valid_out), _ptr(conflict_out)), ctx)


def mrv_clearance(ctx, batch: BatchS, q: int, ts, out):
    _check(lib().mrv_clearance(ctx, C.byref(batch), q, _ptr(ts), len(ts), _ptr(out)), ctx)


def mrv_sync(ctx):
    _check(lib().mrv_sync(ctx), ctx)


def mrv_set_limits(ctx, kernel_budget_ms: float = 0.0):
    _check(lib().mrv_set_limits(ctx, C.byref(Limits(kernel_budget_ms))), ctx)


def mrv_get_stats(ctx) -> dict:
    s = Stats()
    _check(lib().mrv_get_stats(ctx, C.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def mrv_set_tuning(ctx, slices_per_item=1, warps_per_block=4, blocks_per_sm=0, tile_split=4, mv_order=0):
    t = Tuning(slices_per_item, warps_per_block, blocks_per_sm, tile_split, mv_order)
    _check(lib().mrv_set_tuning(ctx, C.byref(t)), ctx)


def mrv_get_tuning(ctx) -> dict:
    t = Tuning()
    _check(lib().mrv_get_tuning(ctx, C.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in Tuning._fields_}


def mrv_autotune(ctx, batch: BatchS, cache_path: Optional[str] = None) -> dict:
    t = Tuning()
    _check(lib().mrv_autotune(ctx, C.byref(batch), None if cache_path is None else str(cache_path).encode(),
                              C.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in Tuning._fields_}


def mrv_graph_create(ctx, batch: BatchS, valid_out, conflict_out):
    g = P()
    _check(lib().mrv_graph_create(ctx, C.byref(batch), _ptr(valid_out), _ptr(conflict_out), C.byref(g)), ctx)
    return g


def mrv_graph_launch(g):
    _check(lib().mrv_graph_launch(g))


def mrv_graph_destroy(g):
    _check(lib().mrv_graph_destroy(g))


# ---------------------------------------------------------------------------
# conveniences
# ---------------------------------------------------------------------------

def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _i32(a):
    return np.ascontiguousarray(a, np.int32)


def robot_desc(m: W.RobotModel, keep: list) -> RobotDesc:
    arrs = [_f32(m.dh), None if m.flange is None else _f32(m.flange), _f32(m.base), _i32(m.sphere_link),
            _f32(m.sphere_xyzr), _i32(m.self_pairs.reshape(-1, 2))]
    keep.extend(a for a in arrs if a is not None)
    dh, fl, base, sl, sx, sp = arrs
    return RobotDesc(m.kind, m.dof, _ptr(dh), _ptr(fl), _ptr(base), m.point_z, sx.shape[0], _ptr(sl), _ptr(sx),
                     sp.shape[0], _ptr(sp) if sp.shape[0] else None)


def env_desc(e: W.Env, keep: list) -> EnvDesc:
    s, b = _f32(e.spheres.reshape(-1, 4)), _f32(e.aabbs.reshape(-1, 6))
    cy = _f32(np.asarray(getattr(e, "cylinders", np.zeros((0, 7)))).reshape(-1, 7))
    keep.extend([s, b, cy])
    return EnvDesc(s.shape[0], _ptr(s) if s.shape[0] else None, b.shape[0], _ptr(b) if b.shape[0] else None,
                   cy.shape[0], _ptr(cy) if cy.shape[0] else None)


class BatchArrays:
    """The CSR arrays of one batch with uploaded ids, on the host (numpy,
    optionally pinned torch tensors) or on the device (torch CUDA tensors)."""

    def __init__(self, arrays: dict, n_queries: int, n_slots: int, n_waypoints: int, wp_stride: int,
                 resolution: float, env_id: int, device: bool):
        self.a = arrays
        self.n_queries, self.n_slots, self.n_waypoints = n_queries, n_slots, n_waypoints
        self.wp_stride, self.resolution, self.env_id, self.device = wp_stride, resolution, env_id, device

    def struct(self, flags: int = 0, with_kind: bool = False, with_env: bool = True) -> BatchS:
        a = self.a
        if self.device:
            flags |= MRV_PTRS_ON_DEVICE
        return BatchS(self.n_queries, self.n_slots, self.n_waypoints, self.env_id, _ptr(a["q_robot_off"]),
                      _ptr(a["slot_robot_id"]), _ptr(a["slot_wp_off"]), _ptr(a["waypoints"]), self.wp_stride,
                      _ptr(a.get("seg_steps")), self.resolution, _ptr(a.get("q_env_id")) if with_env else None,
                      _ptr(a.get("q_kind")) if with_kind else None, flags)

    def to(self, device: str = "cuda", pin: bool = False) -> "BatchArrays":
        import torch
        out = {}
        for k, v in self.a.items():
            if v is None:
                continue
            t = v if not isinstance(v, np.ndarray) else torch.from_numpy(np.ascontiguousarray(v))
            if device == "cpu":
                t = t.cpu()
                out[k] = t.pin_memory() if pin else t
            else:
                out[k] = t.to(device, non_blocking=False).contiguous()
        return BatchArrays(out, self.n_queries, self.n_slots, self.n_waypoints, self.wp_stride, self.resolution,
                           self.env_id, device != "cpu")


class Context:
    """Owns an ``mrv_ctx``; uploads workload models / envs and runs batches."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        self.h = mrv_create(device, stream)
        self._keep: list = []

    def close(self):
        if self.h:
            mrv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload_model(self, m: W.RobotModel) -> int:
        keep: list = []
        return robot_model_upload(self.h, robot_desc(m, keep))

    def upload_env(self, e: W.Env) -> int:
        keep: list = []
        return env_upload(self.h, env_desc(e, keep))

    def bind(self, w: W.Workload, robot_ids=None, env_ids=None) -> BatchArrays:
        """Uploads the workload's models and envs (unless ids are given) and
        returns its batch with slot / env indices mapped to the uploaded ids."""
        if robot_ids is None:
            robot_ids = [self.upload_model(m) for m in w.models]
        if env_ids is None:
            env_ids = [self.upload_env(e) for e in w.envs]
        b = w.batch
        rid = np.asarray(robot_ids, np.int32)
        eid = np.asarray(list(env_ids) + [-1], np.int32)   # index -1 -> id -1
        arrays = {
            "q_robot_off": _i32(b.q_robot_off),
            "slot_robot_id": rid[b.slot_robot],
            "slot_wp_off": _i32(b.slot_wp_off),
            "waypoints": _f32(b.waypoints),
            "seg_steps": None if b.seg_steps is None else _i32(b.seg_steps),
            "q_env_id": None if b.q_env is None else eid[b.q_env],
            "q_kind": None if b.q_kind is None else np.ascontiguousarray(b.q_kind, np.uint8),
        }
        self.robot_ids, self.env_ids = list(robot_ids), list(env_ids)
        env_id = -1 if w.env < 0 else int(eid[w.env])
        return BatchArrays(arrays, b.n_queries, int(b.q_robot_off[-1]), int(b.slot_wp_off[-1]), b.wp_stride,
                           float(b.resolution), env_id, False)

    # -- calls -----------------------------------------------------------------
    def _outs(self, ba: BatchArrays, dtype, shape):
        if ba.device:
            import torch
            tdt = {np.uint8: torch.uint8, np.float32: torch.float32, np.int32: torch.int32}[dtype]
            return torch.empty(shape, dtype=tdt, device="cuda")
        return np.zeros(shape, dtype)

    def mv_validate(self, ba: BatchArrays, check_env: bool = True, exhaustive: bool = False,
                    min_clearance: bool = False, flags: int = 0):
        f = flags | (MRV_CHECK_ENV if check_env else 0) | (MRV_EXHAUSTIVE if exhaustive else 0)
        valid = self._outs(ba, np.uint8, (ba.n_queries,))
        mc = self._outs(ba, np.float32, (ba.n_queries,)) if min_clearance else None
        mv_validate(self.h, ba.struct(f), valid, mc)
        return (valid, mc) if min_clearance else valid

    def ffc_find(self, ba: BatchArrays, exhaustive: bool = False, flags: int = 0):
        f = flags | (MRV_EXHAUSTIVE if exhaustive else 0)
        out = self._outs(ba, np.int32, (ba.n_queries, 3))
        ffc_find(self.h, ba.struct(f), out)
        return out

    def run(self, ba: BatchArrays, check_env: bool = True, exhaustive: bool = False, flags: int = 0):
        f = flags | (MRV_CHECK_ENV if check_env else 0) | (MRV_EXHAUSTIVE if exhaustive else 0)
        valid = self._outs(ba, np.uint8, (ba.n_queries,))
        conf = self._outs(ba, np.int32, (ba.n_queries, 3))
        mrv_run(self.h, ba.struct(f, with_kind=True), valid, conf)
        return valid, conf

    def clearance(self, ba: BatchArrays, q: int, ts, n_spheres: int, check_env: bool = True):
        f = MRV_CHECK_ENV if check_env else 0
        if ba.device:
            import torch
            tts = torch.as_tensor(np.asarray(ts, np.int32), device="cuda")
            out = torch.empty((len(ts), n_spheres), dtype=torch.float32, device="cuda")
        else:
            tts = _i32(ts)
            out = np.zeros((len(ts), n_spheres), np.float32)
        mrv_clearance(self.h, ba.struct(f), q, tts, out)
        return out

    def stats(self) -> dict:
        return mrv_get_stats(self.h)

    def sync(self):
        mrv_sync(self.h)


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

def mrv_server_create(ctx, n_streams=4, device_budget_bytes=1 << 30, max_batch_queries=65536, max_pending=4096):
    o = ServerOpts(n_streams, device_budget_bytes, max_batch_queries, max_pending)
    s = P()
    _check(lib().mrv_server_create(ctx, C.byref(o), C.byref(s)), ctx)
    return s


def mrv_server_destroy(s):
    _check(lib().mrv_server_destroy(s))


def mrv_server_submit(s, batch: BatchS) -> int:
    t = C.c_uint64()
    _check(lib().mrv_server_submit(s, C.byref(batch), C.byref(t)))
    return t.value


def mrv_server_wait(s, ticket: int, timeout_ms: int, valid_out, conflict_out):
    _check(lib().mrv_server_wait(s, ticket, timeout_ms, _ptr(valid_out), _ptr(conflict_out)))


def mrv_server_get_stats(s) -> dict:
    st = ServerStats()
    _check(lib().mrv_server_get_stats(s, C.byref(st)))
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def slice_batch(ba: BatchArrays, q0: int, q1: int) -> BatchArrays:
    """Host BatchArrays holding queries q0..q1-1 of a host batch (offsets
    rebased; arrays are copies)."""
    a = ba.a
    qo = a["q_robot_off"]
    s0, s1 = int(qo[q0]), int(qo[q1])
    so = a["slot_wp_off"]
    w0, w1 = int(so[s0]), int(so[s1])
    out = {"q_robot_off": (qo[q0:q1 + 1] - s0).astype(np.int32),
           "slot_robot_id": a["slot_robot_id"][s0:s1].copy(),
           "slot_wp_off": (so[s0:s1 + 1] - w0).astype(np.int32),
           "waypoints": a["waypoints"][w0:w1].copy(),
           "seg_steps": None if a.get("seg_steps") is None else a["seg_steps"][w0:w1].copy(),
           "q_env_id": None if a.get("q_env_id") is None else a["q_env_id"][q0:q1].copy(),
           "q_kind": None if a.get("q_kind") is None else a["q_kind"][q0:q1].copy()}
    return BatchArrays(out, q1 - q0, s1 - s0, w1 - w0, ba.wp_stride, ba.resolution, ba.env_id, False)


class Server:
    """Continuous-batching request server over a context's resident uploads."""

    def __init__(self, ctx: "Context", n_streams=4, device_budget_bytes=1 << 30, max_batch_queries=65536,
                 max_pending=4096):
        self.ctx = ctx
        self.h = mrv_server_create(ctx.h, n_streams, device_budget_bytes, max_batch_queries, max_pending)

    def submit(self, ba: BatchArrays, check_env=True, exhaustive=False) -> int:
        f = (MRV_CHECK_ENV if check_env else 0) | (MRV_EXHAUSTIVE if exhaustive else 0)
        return mrv_server_submit(self.h, ba.struct(f, with_kind=True))

    def wait(self, ticket: int, n_queries: int, timeout_ms=60000):
        valid = np.zeros(n_queries, np.uint8)
        conf = np.zeros((n_queries, 3), np.int32)
        mrv_server_wait(self.h, ticket, timeout_ms, valid, conf)
        return valid, conf

    def stats(self) -> dict:
        return mrv_server_get_stats(self.h)

    def close(self):
        if self.h:
            mrv_server_destroy(self.h)
            self.h = None
