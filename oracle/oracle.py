"""Python driver of the FP64 scalar oracle (``mrv_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.  It marshals the
seeded workload arrays (numpy, the same FP32 values the CUDA path reads) into
the oracle's own C structs and calls the plain-definition routines: MV
(Alg. 1), FFC (Alg. 2), the first conflict deeper than a bound, decidability margins, per-sphere clearances and the
composite step count (Sec. IV-A3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "mrv_oracle.c"
# MRV_ORACLE_LIB points the driver at another build of the same source (the
# mutation tests use it to check that the pins catch planted mistakes).
LIB = Path(os.environ.get("MRV_ORACLE_LIB", HERE / "liboracle.so"))

_lock = threading.Lock()
_lib = None

JOB_MV, JOB_FFC, JOB_MINCLR, JOB_FFC_DEC, JOB_T, JOB_MV_PRIO, JOB_MINCLR_PRIO, JOB_FFC_BELOW = range(8)


def build(force: bool = False, src: Path = SRC, out: Path = None) -> Path:
    """Compile the oracle with plain gcc (no FMA contraction, no fast-math)."""
    if out is not None:
        subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-pthread", str(src), "-o", str(out), "-lm"], check=True)
        return out
    if "MRV_ORACLE_LIB" in os.environ:
        return LIB
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".so.{os.getpid()}")
        subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-pthread", str(SRC), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


class Robot(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dof", C.c_int32), ("dh", C.c_void_p), ("flange", C.c_void_p),
                ("base", C.c_void_p), ("point_z", C.c_float), ("n_spheres", C.c_int32),
                ("sphere_link", C.c_void_p), ("sphere_xyzr", C.c_void_p), ("n_self", C.c_int32),
                ("self_pairs", C.c_void_p)]


class EnvS(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres", C.c_void_p), ("n_aabbs", C.c_int32),
                ("aabbs", C.c_void_p), ("n_cylinders", C.c_int32), ("cylinders", C.c_void_p)]


class BatchS(C.Structure):
    _fields_ = [("n_queries", C.c_int32), ("q_robot_off", C.c_void_p), ("slot_robot", C.c_void_p),
                ("slot_wp_off", C.c_void_p), ("waypoints", C.c_void_p), ("wp_stride", C.c_int32),
                ("seg_steps", C.c_void_p), ("resolution", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(str(build()))
            P = C.c_void_p
            L.orc_fk.argtypes = [P, P, P]
            L.orc_sphere_sphere.argtypes = [P, C.c_double, P, C.c_double]
            L.orc_sphere_sphere.restype = C.c_double
            L.orc_sphere_box.argtypes = [P, C.c_double, P]
            L.orc_sphere_box.restype = C.c_double
            L.orc_sphere_cylinder.argtypes = [P, C.c_double, P]
            L.orc_sphere_cylinder.restype = C.c_double
            L.orc_query_T.argtypes = [P, P, C.c_int, P]
            L.orc_mv.argtypes = [P, P, P, C.c_int, C.c_int, P]
            L.orc_mv_min_clearance.argtypes = [P, P, P, C.c_int, C.c_int, C.c_double, P]
            L.orc_ffc.argtypes = [P, P, C.c_int, P]
            L.orc_ffc_decidable.argtypes = [P, P, C.c_int, C.c_double, P]
            L.orc_pair_clearances.argtypes = [P, P, C.c_int, C.c_int64, P]
            L.orc_clearance.argtypes = [P, P, P, C.c_int, C.c_int, P, C.c_int, P]
            L.orc_batch_run.argtypes = [C.c_int, P, P, P, P, C.c_int, C.c_int, C.c_double, P, C.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Keep:
    """Holds the contiguous arrays whose pointers were handed to C."""

    def __init__(self):
        self.refs = []

    def arr(self, a, dtype):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(a)
        return a


def _robot_struct(m, keep: _Keep) -> Robot:
    dh = keep.arr(m.dh, np.float32)
    fl = keep.arr(m.flange, np.float32) if m.flange is not None else None
    base = keep.arr(m.base, np.float32)
    sl = keep.arr(m.sphere_link, np.int32)
    sx = keep.arr(m.sphere_xyzr, np.float32)
    sp = keep.arr(m.self_pairs.reshape(-1, 2) if m.self_pairs is not None else np.zeros((0, 2)), np.int32)
    return Robot(m.kind, m.dof, _ptr(dh), _ptr(fl), _ptr(base), m.point_z, sx.shape[0], _ptr(sl), _ptr(sx),
                 sp.shape[0], _ptr(sp))


def _env_struct(e, keep: _Keep) -> EnvS:
    s = keep.arr(e.spheres.reshape(-1, 4), np.float32)
    b = keep.arr(e.aabbs.reshape(-1, 6), np.float32)
    cy = keep.arr(np.asarray(getattr(e, "cylinders", np.zeros((0, 7)))).reshape(-1, 7), np.float32)
    return EnvS(s.shape[0], _ptr(s), b.shape[0], _ptr(b), cy.shape[0], _ptr(cy))


class Oracle:
    """Binds one workload (models, envs, batch) to the C oracle."""

    def __init__(self, w):
        self.w = w
        self.keep = _Keep()
        L = lib()
        self.L = L
        self.robots = (Robot * max(1, len(w.models)))(*[_robot_struct(m, self.keep) for m in w.models])
        self.envs = [_env_struct(e, self.keep) for e in w.envs]
        b = w.batch
        k = self.keep
        qo = k.arr(b.q_robot_off, np.int32)
        sr = k.arr(b.slot_robot, np.int32)
        so = k.arr(b.slot_wp_off, np.int32)
        wp = k.arr(b.waypoints, np.float32)
        st = k.arr(b.seg_steps, np.int32) if b.seg_steps is not None else None
        self.batch = BatchS(b.n_queries, _ptr(qo), _ptr(sr), _ptr(so), _ptr(wp), wp.shape[1], _ptr(st),
                            float(np.float32(b.resolution)) if b.seg_steps is None else 0.0)

    # -- helpers ------------------------------------------------------------
    def _env_of(self, q):
        b = self.w.batch
        e = int(b.q_env[q]) if b.q_env is not None else self.w.env
        return None if e < 0 else self.envs[e]

    def _env_ptrs(self, idx):
        ptrs = (C.c_void_p * max(1, len(idx)))()
        for k, q in enumerate(idx):
            e = self._env_of(int(q))
            ptrs[k] = None if e is None else C.addressof(e)
        return ptrs

    def _run(self, job, idx, out, check_env=True, param=0.0, threads=1):
        idx = np.ascontiguousarray(np.asarray(idx, np.int32))
        envs = self._env_ptrs(idx)
        rc = self.L.orc_batch_run(job, C.byref(self.batch), self.robots, envs, idx.ctypes.data, len(idx),
                                  int(check_env), float(param), out.ctypes.data, int(threads))
        if rc:
            raise ValueError(f"oracle rejected the batch (code {rc})")
        return out

    def _idx(self, idx):
        return np.arange(self.w.batch.n_queries) if idx is None else np.asarray(idx)

    # -- public -------------------------------------------------------------
    def mv(self, idx=None, check_env=None, threads=1, priority=False):
        # priority: the prioritized planner's MV (Sec. IV-C), slot 0 against
        # the obstacles, itself and slots 1..n-1
        idx = self._idx(idx)
        ce = self.w.check_env if check_env is None else check_env
        return self._run(JOB_MV_PRIO if priority else JOB_MV, idx, np.zeros(len(idx), np.uint8), ce,
                         threads=threads)

    def ffc(self, idx=None, threads=1):
        idx = self._idx(idx)
        return self._run(JOB_FFC, idx, np.zeros((len(idx), 3), np.int32), threads=threads)

    def mv_min_clearance(self, idx=None, check_env=None, stop_below=-np.inf, threads=1, priority=False):
        idx = self._idx(idx)
        ce = self.w.check_env if check_env is None else check_env
        return self._run(JOB_MINCLR_PRIO if priority else JOB_MINCLR, idx, np.zeros(len(idx), np.float64), ce,
                         stop_below, threads)

    def ffc_below(self, bound, idx=None, threads=1):
        """First (t, i, j) in Alg. 2's order whose pair clearance is below
        `bound` ((-1, -1, -1) if none); bound 0 is FFC itself."""
        idx = self._idx(idx)
        return self._run(JOB_FFC_BELOW, idx, np.zeros((len(idx), 3), np.int32), param=bound, threads=threads)

    def ffc_decidable(self, idx=None, margin=1e-4, threads=1):
        idx = self._idx(idx)
        return self._run(JOB_FFC_DEC, idx, np.zeros(len(idx), np.uint8), param=margin,
                         threads=threads).astype(bool)

    def query_T(self, idx=None, threads=1):
        idx = self._idx(idx)
        return self._run(JOB_T, idx, np.zeros(len(idx), np.int64), threads=threads)

    def pair_clearances(self, q, t):
        n = int(self.w.batch.q_robot_off[q + 1] - self.w.batch.q_robot_off[q])
        out = np.zeros(max(1, n * (n - 1) // 2), np.float64)
        rc = self.L.orc_pair_clearances(C.byref(self.batch), self.robots, int(q), int(t), out.ctypes.data)
        if rc:
            raise ValueError("oracle rejected the query")
        return out[: n * (n - 1) // 2]

    def clearance(self, q, ts, check_env=None):
        b = self.w.batch
        ce = self.w.check_env if check_env is None else check_env
        s0, s1 = b.q_robot_off[q], b.q_robot_off[q + 1]
        M = sum(self.w.models[b.slot_robot[s]].n_spheres for s in range(s0, s1))
        ts = np.ascontiguousarray(np.asarray(ts, np.int64))
        out = np.zeros((len(ts), M), np.float64)
        e = self._env_of(q)
        rc = self.L.orc_clearance(C.byref(self.batch), self.robots, None if e is None else C.byref(e), int(ce),
                                  int(q), ts.ctypes.data, len(ts), out.ctypes.data)
        if rc:
            raise ValueError("oracle rejected the query")
        return out


def fk(model, q) -> np.ndarray:
    """World sphere centers (m,3) of one robot at configuration q (FP64)."""
    keep = _Keep()
    r = _robot_struct(model, keep)
    qq = np.ascontiguousarray(np.asarray(q, np.float64))
    out = np.zeros((model.n_spheres, 3), np.float64)
    rc = lib().orc_fk(C.byref(r), qq.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError(f"oracle FK rejected the model ({rc})")
    return out


def sphere_sphere(ca, ra, cb, rb) -> float:
    a = np.ascontiguousarray(ca, np.float64)
    b = np.ascontiguousarray(cb, np.float64)
    return lib().orc_sphere_sphere(a.ctypes.data, float(ra), b.ctypes.data, float(rb))


def sphere_box(c, r, box) -> float:
    a = np.ascontiguousarray(c, np.float64)
    bx = np.ascontiguousarray(box, np.float32)
    return lib().orc_sphere_box(a.ctypes.data, float(r), bx.ctypes.data)


def sphere_cylinder(c, r, cyl) -> float:
    """Signed clearance of a sphere and a solid cylinder (a xyz, b xyz, radius)."""
    a = np.ascontiguousarray(c, np.float64)
    cy = np.ascontiguousarray(cyl, np.float32)
    return lib().orc_sphere_cylinder(a.ctypes.data, float(r), cy.ctypes.data)
