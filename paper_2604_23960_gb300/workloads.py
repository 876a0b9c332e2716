"""Seeded synthetic workloads for multi-robot motion validation.

This module only *draws inputs*: robot models (kinematic chains with sphere
sets), obstacle sets and batches of synchronized multi-robot motions.  It holds
none of the validation arithmetic (no forward kinematics of a configuration,
no collision test, no discretisation): the FP64 oracle and the CUDA path both
consume what it produces, and neither is imported here.

Workload shapes follow the paper's experiments (Sec. IV-A): Panda-like 7-DOF
arms approximated by spheres, planar disc robots constrained to a plane, cage
obstacles, random motions with valid endpoints (Sec. IV-A1), a per-timestep
C-space resolution (Sec. IV-A3).  The paper's own scenarios (Panda Cage,
Mobile Cross, Heterogeneous) and the VAMP Panda sphere model are not
available, so seeded stand-ins with the same structure are drawn here.

Data layout shared with the oracle and the C ABI
------------------------------------------------
RobotModel   kind 0 = modified-DH chain, 1 = point robot (dof 2 with fixed z,
             or dof 3); dh rows are (a, alpha, d, theta_offset) per joint;
             sphere_link 0 = base frame, k = frame after joint k, dof+1 =
             flange frame (DH chains only); sphere_xyzr is link-local.
Env          spheres (n,4) world xyzr; aabbs (n,6) lo xyz then hi xyz.
Batch        ragged CSR: q_robot_off (Q+1) -> slots; slot_robot (S) indexes the
             workload's model list; slot_wp_off (S+1) -> waypoints; waypoints
             (W, wp_stride) float32 rows (first dof entries used); seg_steps
             (W,) int32 = interpolation steps from a waypoint to the next one of
             the same slot (entry of a slot's last waypoint unused), or None for
             the start/goal form where the step count follows from
             `resolution`; q_kind (Q,) uint8 0 = MV, 1 = FFC (optional);
             q_env (Q,) int32 index into the env list, -1 = none (optional).

The seeded fixtures that need the method's arithmetic to be drawn (the
self-collision pair list of the Panda-like model and the pools of env+self
valid endpoint configurations) are written by ``oracle/make_cage_fixtures.py``
and stored in ``tests/golden/cage_fixtures.npz``; this module only loads them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from pathlib import Path
from typing import List, Optional

import numpy as np

KIND_DH = 0
KIND_POINT = 1
KIND_MV = 0
KIND_FFC = 1

FIXTURES = Path(__file__).resolve().parents[1] / "tests" / "golden" / "cage_fixtures.npz"


@dataclass
class RobotModel:
    kind: int
    dof: int
    dh: np.ndarray            # (dof,4) float32: a, alpha, d, theta_offset
    flange: Optional[np.ndarray]   # (3,4) float32 or None
    joint_lo: np.ndarray      # (dof,) float32
    joint_hi: np.ndarray      # (dof,) float32
    base: np.ndarray          # (3,4) float32 world <- base
    point_z: float
    sphere_link: np.ndarray   # (m,) int32
    sphere_xyzr: np.ndarray   # (m,4) float32
    self_pairs: np.ndarray    # (k,2) int32
    name: str = ""

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_xyzr.shape[0])


@dataclass
class Env:
    spheres: np.ndarray       # (n,4) float32
    aabbs: np.ndarray         # (n,6) float32
    name: str = ""
    # (n,7) float32: solid cylinders, axis end a xyz, axis end b xyz, radius
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 7), np.float32))


@dataclass
class Batch:
    q_robot_off: np.ndarray
    slot_robot: np.ndarray
    slot_wp_off: np.ndarray
    waypoints: np.ndarray
    seg_steps: Optional[np.ndarray]
    resolution: float = 0.0
    q_kind: Optional[np.ndarray] = None
    q_env: Optional[np.ndarray] = None

    @property
    def n_queries(self) -> int:
        return int(self.q_robot_off.shape[0] - 1)

    @property
    def wp_stride(self) -> int:
        return int(self.waypoints.shape[1])


@dataclass
class Workload:
    name: str
    models: List[RobotModel]
    envs: List[Env]
    batch: Batch
    env: int = -1              # default env index for the whole batch (-1: none)
    check_env: bool = True
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# small constructors
# ---------------------------------------------------------------------------

def _pose(x: float, y: float, z: float, yaw: float = 0.0) -> np.ndarray:
    """3x4 rigid transform Trans(x,y,z) RotZ(yaw) (input synthesis only)."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0, x], [s, c, 0.0, y], [0.0, 0.0, 1.0, z]], np.float32)


def _identity34() -> np.ndarray:
    return _pose(0.0, 0.0, 0.0)


def disc_robot(radius: float = 0.25, z0: float = 0.0, lo=(0.0, 0.0), hi=(10.0, 10.0),
               name: str = "disc") -> RobotModel:
    """Point robot moving in (x, y) at fixed height z0, one sphere of `radius`
    (the paper's mobile robots are spheres constrained to a plane, Sec. IV-A2)."""
    return RobotModel(kind=KIND_POINT, dof=2, dh=np.zeros((2, 4), np.float32), flange=None,
                      joint_lo=np.array(lo, np.float32), joint_hi=np.array(hi, np.float32),
                      base=_identity34(), point_z=float(z0),
                      sphere_link=np.array([1], np.int32),
                      sphere_xyzr=np.array([[0.0, 0.0, 0.0, radius]], np.float32),
                      self_pairs=np.zeros((0, 2), np.int32), name=name)


# Franka Emika Panda kinematics, public datasheet values in Craig's modified DH
# convention: per joint (a_{i-1}, alpha_{i-1}, d_i, theta offset).
PANDA_DH = np.array([
    [0.0, 0.0, 0.333, 0.0],
    [0.0, -math.pi / 2, 0.0, 0.0],
    [0.0, math.pi / 2, 0.316, 0.0],
    [0.0825, math.pi / 2, 0.0, 0.0],
    [-0.0825, -math.pi / 2, 0.384, 0.0],
    [0.0, math.pi / 2, 0.0, 0.0],
    [0.088, math.pi / 2, 0.0, 0.0],
], np.float32)
PANDA_LO = np.array([-2.8973, -1.7628, -2.8973, -3.0718, -2.8973, -0.0175, -2.8973], np.float32)
PANDA_HI = np.array([2.8973, 1.7628, 2.8973, -0.0698, 2.8973, 3.7525, 2.8973], np.float32)
# flange: 0.107 m along z7, hand rotated -pi/4 about z (public datasheet)
PANDA_FLANGE = np.array([[math.cos(-math.pi / 4), -math.sin(-math.pi / 4), 0.0, 0.0],
                         [math.sin(-math.pi / 4), math.cos(-math.pi / 4), 0.0, 0.0],
                         [0.0, 0.0, 1.0, 0.107]], np.float32)
PANDA_HAND_LEN = 0.1034


def _panda_segments():
    """Body segments (link index, start, end) in link-local coordinates.

    A body k spans from the origin of frame k to the origin of frame k+1, which
    in modified DH sits at (a, -sin(alpha) d, cos(alpha) d) of the next joint's
    row, independent of the joint angle; the hand spans the flange frame's z.
    """
    segs = []
    for k in range(8):
        if k < 7:
            a, alpha, d = (float(PANDA_DH[k, 0]), float(PANDA_DH[k, 1]), float(PANDA_DH[k, 2]))
            # row k of the table maps frame k (frame 0 = base) to frame k+1
            end = np.array([a, -math.sin(alpha) * d, math.cos(alpha) * d])
        else:
            end = np.array([0.0, 0.0, 0.107])
        segs.append([k, np.zeros(3), end])
    segs.append([8, np.zeros(3), np.array([0.0, 0.0, PANDA_HAND_LEN])])
    return segs


def panda_like_spheres(seed: int = 102, n_spheres: int = 64):
    """64 seeded spheres along the Panda-like links: at least 4 per body, the
    rest in proportion to segment length; centers on the segment with a jitter
    of at most 0.02 m, radii U(0.03, 0.08)."""
    rng = np.random.default_rng(seed)
    segs = _panda_segments()
    lens = np.array([np.linalg.norm(e - s) for _, s, e in segs])
    nb = len(segs)
    counts = np.full(nb, 4)
    extra = n_spheres - counts.sum()
    share = lens / lens.sum() * extra
    add = np.floor(share).astype(int)
    rem = extra - add.sum()
    order = np.argsort(-(share - add), kind="stable")
    add[order[:rem]] += 1
    counts += add
    links, xyzr = [], []
    for (link, s, e), c in zip(segs, counts):
        for u in (np.arange(c) + 0.5) / c:
            p = s + (e - s) * u
            jit = rng.uniform(-1.0, 1.0, 3)
            jit *= 0.02 * rng.uniform() / max(np.linalg.norm(jit), 1e-12)
            r = rng.uniform(0.03, 0.08)
            links.append(link)
            xyzr.append([p[0] + jit[0], p[1] + jit[1], p[2] + jit[2], r])
    return np.array(links, np.int32), np.array(xyzr, np.float32)


def panda_like(base: np.ndarray, self_pairs: Optional[np.ndarray] = None, seed: int = 102,
               name: str = "panda") -> RobotModel:
    links, xyzr = panda_like_spheres(seed)
    return RobotModel(kind=KIND_DH, dof=7, dh=PANDA_DH.copy(), flange=PANDA_FLANGE.copy(),
                      joint_lo=PANDA_LO.copy(), joint_hi=PANDA_HI.copy(), base=base.astype(np.float32),
                      point_z=0.0, sphere_link=links, sphere_xyzr=xyzr,
                      self_pairs=(np.zeros((0, 2), np.int32) if self_pairs is None
                                  else np.ascontiguousarray(self_pairs, np.int32)), name=name)


CAGE_BASES = [(0.6, 0.6), (-0.6, 0.6), (-0.6, -0.6), (0.6, -0.6)]


def cage_bases() -> List[np.ndarray]:
    """Bases at the corners of a 1.2 m square, yawed to face its center."""
    return [_pose(x, y, 0.0, math.atan2(-y, -x)) for x, y in CAGE_BASES]


def load_cage_fixtures(path: Path = FIXTURES) -> dict:
    if not path.exists():
        raise FileNotFoundError(
            f"{path} missing: run `python oracle/make_cage_fixtures.py` to draw it")
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def cage_arms(fixtures: Optional[dict] = None) -> List[RobotModel]:
    fx = load_cage_fixtures() if fixtures is None else fixtures
    return [panda_like(b, fx["self_pairs"], name=f"panda{k}") for k, b in enumerate(cage_bases())]


CEILING_Z = 2.0
CAGE8_CEILING = [(0.0, 0.85), (-0.85, 0.0), (0.0, -0.85), (0.85, 0.0)]


def _pose_ceiling(x: float, y: float, z: float, yaw: float) -> np.ndarray:
    """3x4 transform Trans(x,y,z) RotZ(yaw) RotX(pi): a base hanging upside
    down from a ceiling at height z (input synthesis only)."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, s, 0.0, x], [s, -c, 0.0, y], [0.0, 0.0, -1.0, z]], np.float32)


def cage8_bases() -> List[np.ndarray]:
    """Cage team of the paper's Cage scenario, floor and ceiling mounted: the
    four floor arms of the 4-arm cage plus four arms hanging from the ceiling
    (z = 2 m) at (0, +-0.85) and (+-0.85, 0), all yawed to face the center."""
    floor = cage_bases()
    ceil = [_pose_ceiling(x, y, CEILING_Z, math.atan2(-y, -x)) for x, y in CAGE8_CEILING]
    return floor + ceil


def cage16_bases() -> List[np.ndarray]:
    """16-arm Cage team (the paper's largest Cage, floor and ceiling mounted):
    the 8-arm team, then floor arms under its four ceiling arms and ceiling
    arms above its four floor arms, so each of the eight positions carries a
    floor and a ceiling arm, all yawed to face the center."""
    floor = [_pose(x, y, 0.0, math.atan2(-y, -x)) for x, y in CAGE8_CEILING]
    ceil = [_pose_ceiling(x, y, CEILING_Z, math.atan2(-y, -x)) for x, y in CAGE_BASES]
    return cage8_bases() + floor + ceil


def load_cage8_fixtures(path: Optional[Path] = None) -> dict:
    path = FIXTURES.parent / "cage8_fixtures.npz" if path is None else path
    if not path.exists():
        raise FileNotFoundError(
            f"{path} missing: run `python oracle/make_cage_fixtures.py --cage8` to draw it")
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def cage8_arms(fixtures: Optional[dict] = None) -> List[RobotModel]:
    fx = load_cage_fixtures() if fixtures is None else fixtures
    return [panda_like(b, fx["self_pairs"], name=f"cage8_arm{k}") for k, b in enumerate(cage8_bases())]


def load_cage16_fixtures(path: Optional[Path] = None) -> dict:
    path = FIXTURES.parent / "cage16_fixtures.npz" if path is None else path
    if not path.exists():
        raise FileNotFoundError(
            f"{path} missing: run `python oracle/make_cage_fixtures.py --cage16` to draw it")
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def cage16_arms(fixtures: Optional[dict] = None) -> List[RobotModel]:
    fx = load_cage_fixtures() if fixtures is None else fixtures
    return [panda_like(b, fx["self_pairs"], name=f"cage16_arm{k}") for k, b in enumerate(cage16_bases())]


# ---------------------------------------------------------------------------
# environments
# ---------------------------------------------------------------------------

def world_boxes(seed: int = 101, n: int = 20, pad: Optional[tuple] = None) -> Env:
    """20 axis-aligned boxes in a 10x10 m world, sides U(0.2, 1.5) per axis,
    centers U(0, 10), spanning z in [-1, 1].  With `pad` = (x0, y0, x1, y1),
    boxes overlapping that rectangle are redrawn."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        c = rng.uniform(0.0, 10.0, 2)
        s = rng.uniform(0.2, 1.5, 2)
        lo, hi = c - s / 2, c + s / 2
        if pad is not None and lo[0] < pad[2] and hi[0] > pad[0] and lo[1] < pad[3] and hi[1] > pad[1]:
            continue
        out.append([lo[0], lo[1], -1.0, hi[0], hi[1], 1.0])
    return Env(np.zeros((0, 4), np.float32), np.array(out, np.float32), name="world")


def cage_env(seed: int = 103) -> Env:
    """Cage: 12 bars of 0.04 m section on the edges of [-1.1,1.1]^2 x [0,1.6]
    plus 40 spheres r ~ U(0.04, 0.10) with centers U([-1,1]^2 x [0.1,1.5]),
    redrawn when within 0.25 m of an arm base's vertical axis."""
    rng = np.random.default_rng(seed)
    h, t, zt = 1.1, 0.02, 1.6
    bars = []
    for x in (-h, h):
        for y in (-h, h):   # vertical posts
            bars.append([x - t, y - t, 0.0, x + t, y + t, zt])
    for z in (0.0, zt):
        for y in (-h, h):   # along x
            bars.append([-h - t, y - t, z - t, h + t, y + t, z + t])
        for x in (-h, h):   # along y
            bars.append([x - t, -h - t, z - t, x + t, h + t, z + t])
    sph = []
    while len(sph) < 40:
        c = rng.uniform([-1.0, -1.0, 0.1], [1.0, 1.0, 1.5])
        r = rng.uniform(0.04, 0.10)
        if min(math.hypot(c[0] - bx, c[1] - by) for bx, by in CAGE_BASES) < 0.25:
            continue
        sph.append([c[0], c[1], c[2], r])
    return Env(np.array(sph, np.float32), np.array(bars, np.float32), name="cage")



def cage_env_cyl(seed: int = 104, n_inner: int = 16) -> Env:
    """Cylinder cage (the paper's Cage obstacles are cylinders): 4 vertical
    posts and 8 beams of radius 0.02 m on the edges of [-1.1,1.1]^2 x [0,2],
    plus `n_inner` cylinders of radius U(0.03, 0.08) and length U(0.2, 0.6)
    with uniformly random axis directions and centers U([-1,1]^2 x [0.2,1.8]),
    redrawn when within 0.3 m of a floor or ceiling arm base's vertical axis."""
    rng = np.random.default_rng(seed)
    h, zt, rb = 1.1, CEILING_Z, 0.02
    cyl = []
    for x in (-h, h):
        for y in (-h, h):
            cyl.append([x, y, 0.0, x, y, zt, rb])
    for z in (0.0, zt):
        for y in (-h, h):
            cyl.append([-h, y, z, h, y, z, rb])
        for x in (-h, h):
            cyl.append([x, -h, z, x, h, z, rb])
    axes = [(x, y) for x, y in CAGE_BASES] + CAGE8_CEILING
    while len(cyl) < 12 + n_inner:
        c = rng.uniform([-1.0, -1.0, 0.2], [1.0, 1.0, 1.8])
        if min(math.hypot(c[0] - x, c[1] - y) for x, y in axes) < 0.3:
            continue
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        half = rng.uniform(0.1, 0.3)
        a, b = c - half * d, c + half * d
        cyl.append([*a, *b, rng.uniform(0.03, 0.08)])
    return Env(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), "cage_cyl",
               np.asarray(cyl, np.float32))

def empty_env() -> Env:
    return Env(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), name="empty")


# ---------------------------------------------------------------------------
# batch assembly
# ---------------------------------------------------------------------------

class BatchBuilder:
    """Accumulates queries (lists of per-slot waypoint arrays) into the CSR layout."""

    def __init__(self, wp_stride: int, timed: bool):
        self.stride = wp_stride
        self.timed = timed
        self.q_off = [0]
        self.slot_robot: list = []
        self.slot_wp_off = [0]
        self.wps: list = []
        self.steps: list = []
        self.kind: list = []
        self.env: list = []

    def add(self, robots, paths, steps=None, kind=KIND_MV, env=-1):
        for s, (r, p) in enumerate(zip(robots, paths)):
            p = np.asarray(p, np.float32)
            if p.ndim == 1:
                p = p[None, :]
            row = np.zeros((p.shape[0], self.stride), np.float32)
            row[:, : p.shape[1]] = p
            self.wps.append(row)
            self.slot_robot.append(r)
            self.slot_wp_off.append(self.slot_wp_off[-1] + p.shape[0])
            if self.timed:
                st = np.zeros(p.shape[0], np.int32)
                if p.shape[0] > 1:
                    st[:-1] = np.asarray(steps[s], np.int32)
                self.steps.append(st)
        self.q_off.append(len(self.slot_robot))
        self.kind.append(kind)
        self.env.append(env)

    def build(self, resolution: float = 0.0) -> Batch:
        wps = np.concatenate(self.wps) if self.wps else np.zeros((0, self.stride), np.float32)
        steps = (np.concatenate(self.steps).astype(np.int32) if self.steps else np.zeros(0, np.int32)) \
            if self.timed else None
        return Batch(np.array(self.q_off, np.int32), np.array(self.slot_robot, np.int32),
                     np.array(self.slot_wp_off, np.int32), np.ascontiguousarray(wps), steps,
                     float(resolution), np.array(self.kind, np.uint8), np.array(self.env, np.int32))


def _fast_batch(n_q: int, n_robot: int, slot_robot: np.ndarray, wps: np.ndarray,
                steps: Optional[np.ndarray], resolution: float, kind, env) -> Batch:
    """Vectorised CSR assembly for batches with a fixed robot count per query
    and a fixed waypoint count per slot."""
    n_slots = n_q * n_robot
    n_wp = wps.shape[0] // n_slots
    return Batch(np.arange(0, n_slots + 1, n_robot, dtype=np.int32),
                 slot_robot.astype(np.int32),
                 np.arange(0, n_slots * n_wp + 1, n_wp, dtype=np.int32),
                 np.ascontiguousarray(wps, np.float32),
                 None if steps is None else np.ascontiguousarray(steps, np.int32),
                 float(resolution),
                 np.broadcast_to(np.asarray(kind, np.uint8), (n_q,)).copy(),
                 np.broadcast_to(np.asarray(env, np.int32), (n_q,)).copy())


# ---------------------------------------------------------------------------
# the five workload configurations
# ---------------------------------------------------------------------------

def make_plain_discs(n_queries: int = 1000, env_seed: int = 101, query_seed: int = 201,
                     kind: int = KIND_MV) -> Workload:
    """Two planar disc robots (r = 0.25 m) in a 10x10 m world with 20 boxes;
    straight start->goal motions drawn uniformly; resolution 0.05 m."""
    models = [disc_robot(0.25, 0.0, name="disc0"), disc_robot(0.25, 0.0, name="disc1")]
    env = world_boxes(env_seed)
    rng = np.random.default_rng(query_seed)
    pts = rng.uniform(0.0, 10.0, (n_queries, 2, 2, 2)).astype(np.float32)  # q, robot, start/goal, xy
    wps = pts.reshape(-1, 2)
    slot_robot = np.tile(np.arange(2), n_queries)
    b = _fast_batch(n_queries, 2, slot_robot, wps, None, 0.05, kind, 0)
    return Workload("plain_discs", models, [env], b, env=0, check_env=True,
                    meta={"robots": 2, "resolution": 0.05})


def make_cage_mv(n_queries: int = 10000, query_seed: int = 203, fixtures: Optional[dict] = None,
                 env_seed: int = 103) -> Workload:
    """4 Panda-like arms in the cage; composite start->goal joint-space motions
    whose endpoints are drawn from per-arm pools of env+self valid
    configurations; resolution 1/32 rad."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    models = cage_arms(fx)
    env = cage_env(env_seed)
    rng = np.random.default_rng(query_seed)
    pools = fx["endpoint_pool"]                     # (4, P, 7)
    P = pools.shape[1]
    idx = rng.integers(0, P, (n_queries, 4, 2))
    cfg = pools[np.arange(4)[None, :, None], idx]   # (Q, 4, 2, 7)
    wps = cfg.reshape(-1, 7)
    slot_robot = np.tile(np.arange(4), n_queries)
    b = _fast_batch(n_queries, 4, slot_robot, wps, None, 1.0 / 32.0, KIND_MV, 0)
    return Workload("cage_mv", models, [env], b, env=0, check_env=True,
                    meta={"robots": 4, "resolution": 1.0 / 32.0})


def make_cage_ffc(n_queries: int = 100000, query_seed: int = 204, fixtures: Optional[dict] = None,
                  wp_range=(20, 60), step_range=(8, 64)) -> Workload:
    """4 arms, independent timed paths: 20-60 waypoints uniform in the joint
    limits and 8-64 interpolation steps per segment; shorter paths are padded
    with their last configuration (Sec. III-A)."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    models = cage_arms(fx)
    rng = np.random.default_rng(query_seed)
    n_wp = rng.integers(wp_range[0], wp_range[1] + 1, (n_queries, 4))
    tot = int(n_wp.sum())
    wps = rng.uniform(PANDA_LO, PANDA_HI, (tot, 7)).astype(np.float32)
    steps = rng.integers(step_range[0], step_range[1] + 1, tot).astype(np.int32)
    slot_wp_off = np.zeros(n_queries * 4 + 1, np.int32)
    np.cumsum(n_wp.reshape(-1), out=slot_wp_off[1:])
    steps[slot_wp_off[1:] - 1] = 0          # a slot's last waypoint has no outgoing segment
    b = Batch(np.arange(0, n_queries * 4 + 1, 4, dtype=np.int32),
              np.tile(np.arange(4, dtype=np.int32), n_queries), slot_wp_off, wps, steps, 0.0,
              np.full(n_queries, KIND_FFC, np.uint8), np.full(n_queries, -1, np.int32))
    return Workload("cage_ffc", models, [], b, env=-1, check_env=False,
                    meta={"robots": 4})


def make_cage_priority(n_queries: int = 10000, query_seed: int = 207, fixtures: Optional[dict] = None,
                       env_seed: int = 103, seg_range=(1, 3)) -> Workload:
    """Edge checks of prioritized planning (Sec. IV-C) in the cage: per query
    one arm (slot 0, drawn uniformly) moves along a start->goal edge between
    env+self valid configurations at 1/32 rad per step (L steps), and the
    three other arms (slots 1..3, higher priority) follow timed paths of 1-3
    segments through valid configurations spanning the same L steps.  To be
    run with MRV_PRIORITY: slot 0 against the cage, itself and slots 1..3."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    models = cage_arms(fx)
    env = cage_env(env_seed)
    rng = np.random.default_rng(query_seed)
    pools = fx["endpoint_pool"]                      # (4, P, 7)
    P = pools.shape[1]
    cur = rng.integers(0, 4, n_queries)
    wps, steps, slot_robot, slot_wp_off = [], [], [], [0]
    for q in range(n_queries):
        c = int(cur[q])
        s, g = pools[c, rng.integers(0, P, 2)]
        d = float(np.linalg.norm(g.astype(np.float64) - s.astype(np.float64)))
        L = max(1, math.ceil(d * 32.0))
        order = [c] + [a for a in range(4) if a != c]
        for k, a in enumerate(order):
            if k == 0:
                path, st = [s, g], [L]
            else:
                ns = int(rng.integers(seg_range[0], seg_range[1] + 1))
                ns = min(ns, L)
                cuts = np.sort(rng.choice(np.arange(1, L), ns - 1, replace=False)) if ns > 1 else np.zeros(0, int)
                st = list(np.diff(np.concatenate([[0], cuts, [L]])).astype(int))
                path = list(pools[a, rng.integers(0, P, ns + 1)])
            wps.extend(path)
            steps.extend(st + [0])
            slot_robot.append(a)
            slot_wp_off.append(slot_wp_off[-1] + len(path))
    b = Batch(np.arange(0, n_queries * 4 + 1, 4, dtype=np.int32), np.asarray(slot_robot, np.int32),
              np.asarray(slot_wp_off, np.int32), np.asarray(wps, np.float32).reshape(-1, 7),
              np.asarray(steps, np.int32), 0.0, np.full(n_queries, KIND_MV, np.uint8),
              np.zeros(n_queries, np.int32))
    return Workload("cage_priority", models, [env], b, env=0, check_env=True,
                    meta={"robots": 4, "priority": True})


def make_cage8_mv(n_queries: int = 10000, query_seed: int = 208, fixtures: Optional[dict] = None,
                  fixtures8: Optional[dict] = None) -> Workload:
    """MV for the floor- and ceiling-mounted 8-arm team in the cylinder cage:
    composite start->goal motions whose endpoints come from per-arm pools of
    env+self valid configurations; resolution 1/32 rad."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    f8 = load_cage8_fixtures() if fixtures8 is None else fixtures8
    models = cage8_arms(fx)
    env = cage_env_cyl()
    rng = np.random.default_rng(query_seed)
    pools = f8["endpoint_pool"]                      # (8, P, 7)
    P = pools.shape[1]
    idx = rng.integers(0, P, (n_queries, 8, 2))
    cfg = pools[np.arange(8)[None, :, None], idx]    # (Q, 8, 2, 7)
    b = _fast_batch(n_queries, 8, np.tile(np.arange(8), n_queries), cfg.reshape(-1, 7), None, 1.0 / 32.0,
                    KIND_MV, 0)
    return Workload("cage8_mv", models, [env], b, env=0, check_env=True,
                    meta={"robots": 8, "resolution": 1.0 / 32.0})


def make_cage16_mv(n_queries: int = 10000, query_seed: int = 209, fixtures: Optional[dict] = None,
                   fixtures16: Optional[dict] = None, edge: Optional[float] = 0.5) -> Workload:
    """MV for the floor- and ceiling-mounted 16-arm team in the cylinder cage
    (Sec. V-A, Fig. 3b), on planner-like edges: each motion starts at a
    whole-team configuration that is valid (every arm env+self valid and clear
    of the others) and heads for another one, cut to at most `edge` rad of
    C-space distance for the arm that moves furthest (a tree planner's
    extension range; None: the whole way); resolution 1/32 rad.  1024 spheres
    per query: the large-team kernel.  At 0.5 rad about 15% of the edges are
    valid and T is about 16; whole motions between two team configurations
    are almost never valid."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    f16 = load_cage16_fixtures() if fixtures16 is None else fixtures16
    models = cage16_arms(fx)
    env = cage_env_cyl()
    rng = np.random.default_rng(query_seed)
    team = f16["team_states"]                        # (K, 16, 7)
    K = team.shape[0]
    a = rng.integers(0, K, n_queries)
    b = (a + rng.integers(1, K, n_queries)) % K      # a different configuration
    start = team[a].astype(np.float64)
    d = team[b].astype(np.float64) - start
    if edge is not None:
        reach = np.linalg.norm(d, axis=2).max(axis=1)
        d *= np.minimum(1.0, edge / np.maximum(reach, 1e-12))[:, None, None]
    cfg = np.stack([team[a], (start + d).astype(np.float32)], axis=2)   # (Q, 16, 2, 7)
    bt = _fast_batch(n_queries, 16, np.tile(np.arange(16), n_queries), cfg.reshape(-1, 7), None, 1.0 / 32.0,
                     KIND_MV, 0)
    return Workload("cage16_mv", models, [env], bt, env=0, check_env=True,
                    meta={"robots": 16, "resolution": 1.0 / 32.0, "edge": edge})


def make_cage16_ffc(n_queries: int = 10000, query_seed: int = 210, fixtures: Optional[dict] = None,
                    fixtures16: Optional[dict] = None) -> Workload:
    """FFC on the 16-arm team's whole motions between two valid team
    configurations (120 robot pairs per state), obstacles ignored (Alg. 2)."""
    w = make_cage16_mv(n_queries, query_seed, fixtures, fixtures16, edge=None)
    w.batch.q_kind = np.full(n_queries, KIND_FFC, np.uint8)
    w.name = "cage16_ffc"
    w.check_env = False
    return w


def make_cage_team_study(n_arms: int, n_queries: int = 500, query_seed: int = 211, obstacles: bool = True,
                         fixtures: Optional[dict] = None, fixtures16: Optional[dict] = None) -> Workload:
    """The validation study's motions (Sec. V-B: 500 random Cage motions with
    valid endpoints for 4, 8 and 16 Pandas, with and without obstacles): the
    first n_arms arms of the 16-arm team (4: the floor corners; 8: the
    floor- and ceiling-mounted 8-arm team), whole motions between two of the
    whole-team valid configurations restricted to those arms (a valid team
    stays valid without some of its arms); resolution 1/32 rad; the cylinder
    cage, or no obstacles (self and robot-robot checks only)."""
    if n_arms not in (4, 8, 16):
        raise ValueError("n_arms must be 4, 8 or 16")
    fx = load_cage_fixtures() if fixtures is None else fixtures
    f16 = load_cage16_fixtures() if fixtures16 is None else fixtures16
    models = cage16_arms(fx)[:n_arms]
    team = f16["team_states"][:, :n_arms]            # (K, n_arms, 7)
    K = team.shape[0]
    rng = np.random.default_rng(query_seed + n_arms)
    a = rng.integers(0, K, n_queries)
    b = (a + rng.integers(1, K, n_queries)) % K
    cfg = np.stack([team[a], team[b]], axis=2)       # (Q, n_arms, 2, 7)
    bt = _fast_batch(n_queries, n_arms, np.tile(np.arange(n_arms), n_queries), cfg.reshape(-1, 7), None,
                     1.0 / 32.0, KIND_MV, 0 if obstacles else -1)
    envs = [cage_env_cyl()] if obstacles else []
    return Workload(f"cage{n_arms}_study{'_obst' if obstacles else ''}", models, envs, bt,
                    env=0 if obstacles else -1, check_env=True,
                    meta={"robots": n_arms, "obstacles": obstacles, "resolution": 1.0 / 32.0})


TEAM_ARM_BASES = [(4.4, 5.0, 0.0), (5.6, 5.0, math.pi)]
TEAM_PAD = (3.8, 3.8, 6.2, 6.2)


def team_models(fixtures: Optional[dict] = None) -> List[RobotModel]:
    """Two arms facing each other at (4.4,5) and (5.6,5) plus a disc model
    (r = 0.25 m at z = 0.25) used for the 2-6 mobile robots."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    arms = [panda_like(_pose(x, y, z=0.0, yaw=yaw), fx["self_pairs"], name=f"team_arm{k}")
            for k, (x, y, yaw) in enumerate(TEAM_ARM_BASES)]
    return arms + [disc_robot(0.25, 0.25, name="team_disc")]


def make_ragged_teams(n_queries: int = 1_000_000, seed: int = 205, fixtures: Optional[dict] = None,
                      len_range=(8, 512)) -> Workload:
    """Heterogeneous ragged batch: the 2 arms plus 0-6 discs per query (2-8
    robots in total), one straight segment per robot with a step count
    L ~ logU[8, 512] shared by the query, MV or FFC with probability 1/2."""
    models = team_models(fixtures)
    env = world_boxes(101, pad=TEAM_PAD)
    rng = np.random.default_rng(seed)
    n_disc = rng.integers(0, 7, n_queries)          # 0..6 discs -> 2..8 robots
    n_rob = 2 + n_disc
    L = np.exp(rng.uniform(math.log(len_range[0]), math.log(len_range[1]), n_queries))
    L = np.clip(np.round(L).astype(np.int32), len_range[0], len_range[1])
    kind = rng.integers(0, 2, n_queries).astype(np.uint8)
    n_slots = int(n_rob.sum())
    q_off = np.zeros(n_queries + 1, np.int32)
    np.cumsum(n_rob, out=q_off[1:])
    slot_idx = np.arange(n_slots) - np.repeat(q_off[:-1], n_rob)
    slot_robot = np.where(slot_idx < 2, slot_idx, 2).astype(np.int32)
    wps = np.zeros((2 * n_slots, 8), np.float32)
    arm = slot_idx < 2
    n_arm = int(arm.sum())
    arm_cfg = rng.uniform(PANDA_LO, PANDA_HI, (n_arm, 2, 7)).astype(np.float32)
    disc_cfg = rng.uniform(0.0, 10.0, (n_slots - n_arm, 2, 2)).astype(np.float32)
    w = wps.reshape(n_slots, 2, 8)
    w[arm, :, :7] = arm_cfg
    w[~arm, :, :2] = disc_cfg
    steps = np.zeros((n_slots, 2), np.int32)
    steps[:, 0] = np.repeat(L, n_rob)
    b = Batch(q_off, slot_robot, np.arange(0, 2 * n_slots + 1, 2, dtype=np.int32), wps,
              steps.reshape(-1), 0.0, kind, np.zeros(n_queries, np.int32))
    return Workload("ragged_teams", models, [env], b, env=0, check_env=True,
                    meta={"len_range": len_range})


def subset(w: Workload, idx) -> Workload:
    """Workload restricted to the queries `idx` (same models and envs)."""
    b = w.batch
    idx = np.asarray(idx, np.int64)
    bb = BatchBuilder(b.wp_stride, b.seg_steps is not None)
    for q in idx:
        s0, s1 = b.q_robot_off[q], b.q_robot_off[q + 1]
        robots, paths, steps = [], [], []
        for s in range(s0, s1):
            w0, w1 = b.slot_wp_off[s], b.slot_wp_off[s + 1]
            robots.append(int(b.slot_robot[s]))
            paths.append(b.waypoints[w0:w1])
            if b.seg_steps is not None:
                steps.append(b.seg_steps[w0:w1 - 1])
        bb.add(robots, paths, steps if b.seg_steps is not None else None,
               int(b.q_kind[q]) if b.q_kind is not None else KIND_MV,
               int(b.q_env[q]) if b.q_env is not None else w.env)
    nb = bb.build(b.resolution)
    return Workload(w.name + f"[{len(idx)}]", w.models, w.envs, nb, w.env, w.check_env, dict(w.meta))


# ---------------------------------------------------------------------------
# serving: four request families over four resident environments
# ---------------------------------------------------------------------------

def make_serving_families(n_per_family: int = 20000, seed: int = 206, fixtures: Optional[dict] = None,
                          len_range=(8, 512)):
    """Four query families sharing one model list and one env list, all in
    the timed form with one segment per robot and L ~ logU[8, 512] steps:
    0: 2-8 discs in the box world; 1: 2-4 cage arms (valid endpoints) in the
    cage; 2: 2-4 cage arms without obstacles; 3: the ragged teams in the
    padded box world.  Queries are MV or FFC with probability 1/2.
    Returns (models, envs, [Workload per family])."""
    fx = load_cage_fixtures() if fixtures is None else fixtures
    arms = cage_arms(fx)
    team = team_models(fx)
    disc = disc_robot(0.25, 0.0, name="disc")
    models = arms + team + [disc]            # 0-3 cage arms, 4-5 team arms, 6 team disc, 7 disc
    envs = [world_boxes(101), cage_env(103), empty_env(), world_boxes(101, pad=TEAM_PAD)]
    rng = np.random.default_rng(seed)
    pools = fx["endpoint_pool"]
    fams = []
    for f in range(4):
        bb = BatchBuilder(8, True)
        for _ in range(n_per_family):
            L = int(np.clip(round(math.exp(rng.uniform(math.log(len_range[0]), math.log(len_range[1])))),
                            len_range[0], len_range[1]))
            kind = int(rng.integers(0, 2))
            if f == 0:
                n = int(rng.integers(2, 9))
                robots = [7] * n
                paths = [rng.uniform(0.0, 10.0, (2, 2)) for _ in range(n)]
            elif f in (1, 2):
                n = int(rng.integers(2, 5))
                robots = sorted(rng.choice(4, n, replace=False).tolist())
                if f == 1:
                    paths = [pools[r][rng.integers(0, pools.shape[1], 2)] for r in robots]
                else:
                    paths = [rng.uniform(PANDA_LO, PANDA_HI, (2, 7)) for _ in robots]
            else:
                nd = int(rng.integers(0, 7))
                robots = [4, 5] + [6] * nd
                paths = [rng.uniform(PANDA_LO, PANDA_HI, (2, 7)) for _ in range(2)] + \
                        [rng.uniform(0.0, 10.0, (2, 2)) for _ in range(nd)]
            bb.add(robots, paths, [[L]] * len(robots), kind, f if f != 2 else -1)
        fams.append(Workload(f"serve{f}", models, envs, bb.build(), env=-1, check_env=True))
    return models, envs, fams
