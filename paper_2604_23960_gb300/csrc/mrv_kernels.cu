// Kernels of multi-robot MotionValidation (MV, Alg. 1) and FindFirstConflict
// (FFC, Alg. 2) for sm_103a.
//
// Work decomposition
//   tile   32 states of one query, the GPU's batch of W = 32 timesteps
//          (PackCfgBatch, Sec. III-A): MV packs them with the rake order
//          t = b + nb*l (nb = ceil((T+1)/32)), FFC (and MV with MRV_LINEAR)
//          with the linear order t = 32b + l.
//   slice  a tile cut into `split` parts: MV slice p takes the rake lanes
//          l = p, p+split, ... (still spread over the whole motion) and visits
//          them from the middle outwards; FFC slice p takes consecutive states
//          in order.  Point-robot queries keep whole tiles (split 1, one lane
//          per state).
//   item   `cte` consecutive slices of one query, walked in order by one warp
//          that stops once the query is decided (MV: any collision; FFC: a
//          conflict at an earlier state).  Items are claimed 1..32 at a time
//          from a global counter in level order (every query's first item,
//          then every query's second item, ...); a claim's lanes check the
//          claimed items' verdicts in parallel, and only undecided ones run.
//   phase  hierarchical MV (Alg. 1, hierarchical branch) runs every slice
//          twice: first the robot-obstacle + self checks, then the pairs.
//   class  queries of up to 8 robots and 512 spheres (class 0) run on the
//          team layout of per-warp shared memory, 12 warps per SM; larger
//          ones, up to 16 robots and 1024 spheres (the 16-arm Cage team),
//          on the large-team layout; k_main is instantiated per layout and
//          each instance takes its class's items (own levels and counter).
// Two per-query flavors:
//   A  (point robots, <= 16 spheres): lane l owns state t(l) of the tile and
//      runs every check of that state; a ballot finds the first conflicting
//      lane.
//   B  (kinematic chains): the warp walks a slice's states; per FK round up
//      to 8 (state, robot) chains (16 for a 16-robot team) run on three lanes
//      each (one row of the link frames per lane, ten chains at a time) into
//      shared memory.  Per state (broadphase path, the
//      default): frame bounding spheres; obstacles from the grid cell of each
//      frame, self-pair groups and frame pairs of other robots go to
//      candidate lists; only the named frames' spheres are placed; the lists
//      are resolved over all lanes (self pairs as row-mask blocks).  With
//      MRV_NO_BROADPHASE every sphere pair is tested (dense path, below).
//
// Sphere-pair test of the dense path.  With centers p relative to an origin
// near the query and k = |p|^2 - r^2, two spheres overlap iff
//     u = k_b - 2 p_a.p_b - 2 r_a r_b  <  -k_a
// (the expanded |p_a - p_b|^2 < (r_a + r_b)^2): four FMAs per test and one
// running minimum per row.  The rounding error of u and k is below
// 24 u (C^2 + rho^2) (C: largest |p|, rho: largest radius, u = 2^-24);
// a row whose minimum falls within twice that band of -k_a is decided again
// by the direct formula, so decisions are those of the direct FP32 formula
// wherever the two could differ.  The broadphase path uses the direct formula.
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include <mutex>

#include "mrv_dev.h"

namespace mrv {

// Index checks of the MRV_CHECKED build (see MRV_CHECK_SITES): CK(i, n, site,
// err) is i when 0 <= i < n; otherwise the first failure's site, index and
// extent go to the error record err[0..3] and the access is redirected to
// element 0 (in bounds), so the kernel never faults and runs to its end.  In
// the normal build CK(i, ...) is i.
#ifdef MRV_CHECKED
__device__ __noinline__ void ck_fail(uint32_t *err, uint32_t site, long long i, long long n) {
  if (atomicCAS(err + 1, 0u, site) == 0u) {
    err[2] = (uint32_t)i;
    err[3] = (uint32_t)n;
  }
  atomicOr(err, kErrChecked);
}
__device__ __forceinline__ long long ck_idx(long long i, long long n, uint32_t site, uint32_t *err) {
  if (i >= 0 && i < n) return i;
  ck_fail(err, site, i, n);
  return 0;
}
#define CK(i, n, site, err) ((decltype((i) + 0))::mrv::ck_idx((long long)(i), (long long)(n), ::mrv::kCk_##site, (err)))
// the half-open range [lo, hi) lies in 0..n-1 (an empty range always does)
#define CK_RANGE(lo, hi, n, site, err)                  \
  do {                                                  \
    if ((hi) > (lo)) {                                  \
      (void)CK((lo), (n), site, (err));                 \
      (void)CK((hi) - 1, (n), site, (err));             \
    }                                                   \
  } while (0)
#else
#define CK(i, n, site, err) (i)
#define CK_RANGE(lo, hi, n, site, err) ((void)0)
#endif

constexpr int kSlotWords = 30;                   // words per RobotSlot in shared memory
constexpr float kEpsU = 48.0f / 16777216.0f;     // 2 x 24 unit roundoffs

struct RobotSlot {           // per-warp staged view of one robot of the query
  const float4 *spheres;
  const int32_t *links;
  const uint32_t *self;      // packed pairs x | y << 16, padded to a multiple of 4
  const int4 *rects;         // self pairs as rectangles (rows x0..x1, columns y0..y1)
  const ModelDev *md;        // the model (frame ranges, bounding spheres, groups)
  const uint32_t *masks;     // self-pair block row masks (null: none)
  int32_t mdl, m, dof, kind, n_self, w0, w1, n_rects;
  int32_t n_links, n_groups;
  int16_t ls[kMaxLinks + 2]; // frame ranges of the sorted spheres (copy of md->link_start)
  int16_t nfr;               // frames holding spheres (bits of md->frame_mask)
};
static_assert(sizeof(RobotSlot) <= kSlotWords * 4, "slot size");

struct TileCtx {
  uint32_t *err;             // the call's error record (index checks of MRV_CHECKED)
  int q, T, n, M, nb, ffc, check_env, exhaustive, broad;
  int lin;                   // linear state order (FFC, or MV with MRV_LINEAR)
  int prio;                  // prioritized MV: slot 0 against obstacles, itself and slots 1..n-1
  int env_rows;              // spheres with obstacle checks: [0, env_rows)
  int self_robots;           // robots with self checks: [0, self_robots)
  int pair_robots;           // robots i whose pairs (i, j > i) are checked
  int self_blk;              // every robot's self pairs come as blocks
  int pr0, pr1;              // robot-pair table entries checked in the current phase
  int fpt;                   // frame-pair table: 0 not used (too many pairs), 1 not built yet, 2 built
  int clr;                   // minimum clearance wanted (full instance only)
  int nef, nef_env;          // frame slots holding spheres (ef): all robots', the obstacle-checked robots'
  int first_phase;           // the current phase is the first visit of its states
  long long rangetests;      // sphere tests per state of the entries pr0..pr1-1
  int split, spt, nslices;
  int env_ns, env_nb;
  const float4 *env_s;
  const float *env_k;
  const float4 *box_lo, *box_hi;
  const EnvDev *env;         // the query's obstacle set (null: none)
  float env_c2, env_r2, rho2;
  long long pairtests, envtests, boxtests, cyltests;
  unsigned long long tests, btests, states, chains, placed, ctests;
  int env_nc;                // obstacle cylinders of the query's env
  const float4 *cyl_a, *cyl_u;
};

constexpr int kCand = 64;        // broadphase candidates per list and state

// Candidates of one state found by the bounding-sphere tests, and the frames
// whose spheres must be placed to resolve them (bit k of need/placed = frame
// slot k = robot k / kMaxLinks, frame k % kMaxLinks), for queries of up to NR
// robots (frame slots < 256).
template <int NR>
struct Cands {
  static constexpr int kWords = (NR * kMaxLinks + 31) / 32;   // frame-slot mask words
  uint32_t pc[kCand];        // robot-robot: frame slot k << 8 | frame slot k2
  uint32_t ec[kCand];        // frame slot << 24 | obstacle sphere
  uint32_t bc[kCand];        // frame slot << 24 | obstacle box
  uint32_t sc[kCand];        // self-pair group: robot << 16 | its first pair
  uint16_t scn[kCand];       // ... and its pair count (blocks: first row mask)
  uint8_t sck[kCand];        // blocks: frame slot of the column frame
  int32_t pf[kCand + 1];     // exclusive prefix of the tests of the list being resolved
  uint32_t yc[kCand];        // frame slot << 24 | obstacle cylinder
  int32_t np, ne, nb, ns, overflow, ny;
  uint32_t need[kWords], placed[kWords];
  // large teams (NR > kTeamRobots): robot-level cull of the robot-robot
  // phase.  Per robot a sphere enclosing its frame bounding spheres at the
  // state; the phase's pair-table entries whose robot spheres overlap; the
  // exclusive prefix of their frame-pair counts.
  static constexpr int kCullR = NR > kTeamRobots ? NR : 1;
  static constexpr int kCullP = NR > kTeamRobots ? NR * (NR - 1) / 2 : 1;
  float4 rsph[kCullR];
  int16_t kept[kCullP];
  int32_t keptf[kCullP + 1];
};

// Per-warp shared memory of the persistent kernel for queries of up to NR
// robots and MQ spheres.  Three layouts are instantiated, one per work class:
// small teams (8 robots, 256 spheres; 16 warps share an SM), teams (8 robots,
// 512 spheres; 12 warps) and large teams (16 robots, 1024 spheres).  Obstacles
// are read through L1 (a per-warp copy of the first obstacles measured the
// same and cost 2.3 KB of every warp's shared memory).
template <int NR, int MQ>
struct WarpSmemT {
  static constexpr int kRobots = NR, kSpheres = MQ;
  static constexpr int kClass = work_class(NR, MQ);
  static constexpr bool kLarge = kClass == 2;   // robot-level cull, self groups in batches
  // threads per SM the instance is compiled for (the register budget)
  static constexpr int kMaxThreads = kClass == 0 ? 512 : 384;
  static constexpr int kChains = NR > kFkChains ? NR : kFkChains;   // FK chains held at once
  using Cl = Cands<NR>;
  TileCtx ctx;               // the current work item's query parameters
  RobotSlot rs[NR];
  int32_t off[NR + 1];
  int32_t seg[NR];           // per robot: waypoint index of the segment of the
                             // latest FK round (states grow within a slice)
  // slots of a single segment (two waypoints: every start/goal slot): the
  // segment's end time (-1: several segments, interpolated from global
  // memory) and its two waypoints, staged once per work item so that an FK
  // round interpolates without waiting on global loads
  int32_t itau[NR];
  alignas(16) float ia[NR][MRV_MAX_DOF];
  alignas(16) float ig[NR][MRV_MAX_DOF];
  float ox, oy, oz;          // origin of the relative frame (world)
  int32_t pad[4];
  // robot pairs i < j of the query, i | j << 4 | n_links_j << 8 | m << 16
  // with m = ceil(4096 / n_links_j) (frame pair g of the pair is (g m >> 12,
  // g mod n_links_j), exact for g < 100), and the exclusive prefix of their
  // frame-pair counts n_links_i x n_links_j
  uint32_t rp[NR * (NR - 1) / 2];
  int16_t rpf[NR * (NR - 1) / 2 + 2];
  // small teams: the query's frame pairs whose two frames hold spheres,
  // frame slot k | k2 << 8, grouped by robot-pair table entry (fpf: the
  // exclusive prefix of their counts per entry); built when a work item first
  // reaches its robot-robot checks
  static constexpr int kFPCap = (NR <= kTeamRobots && MQ <= kSmallSpheres) ? 512 : 0;
  uint16_t fp[kFPCap > 0 ? kFPCap : 1];
  int16_t fpf[NR * (NR - 1) / 2 + 2];
  float4 BS[NR * kMaxLinks];  // per (robot, frame) bounding sphere at the
                              // current state (center relative to o; w < 0: none)
  uint8_t ef[NR * kMaxLinks]; // the query's frame slots holding spheres, by robot
                              // (the others' BS entries stay w < 0 for the item)
  union {
    struct {
      float xf[kChains * kMaxLinks * 12];   // link frames of one FK round
      float4 P[MQ];                         // centers relative to o, radius
      union {
        float K[MQ];                        // dense path: |p|^2 - r^2
        Cl cl;                              // broadphase: candidate lists
      };
    } b;
    float4 PA[kFlavorAMaxSpheres * kWarp];  // flavor A: world centers per lane
  } u;
  static_assert(NR <= 16 && NR * kMaxLinks < 256, "robot and frame-slot indices fit their fields");
};
using WarpSmemSmall = WarpSmemT<kTeamRobots, kSmallSpheres>;
using WarpSmemTeam = WarpSmemT<kTeamRobots, kTeamSpheres>;
using WarpSmemLarge = WarpSmemT<MRV_MAX_ROBOTS, MRV_MAX_QUERY_SPHERES>;
static_assert(WarpSmemSmall::kClass == 0 && WarpSmemTeam::kClass == 1 && WarpSmemLarge::kClass == 2, "classes");

template <class WS>
__host__ __device__ constexpr size_t warp_smem_bytes() { return (sizeof(WS) + 15) & ~size_t(15); }
// small-team layout: 16 warps (4 blocks of 4) must fit the SM's 228 KB with 1 KB reserved per block
static_assert(16 * warp_smem_bytes<WarpSmemSmall>() + 4 * 1024 <= 233472, "shared memory per warp");
// team layout: 12 warps (3 blocks of 4)
static_assert(12 * warp_smem_bytes<WarpSmemTeam>() + 3 * 1024 <= 233472, "shared memory per warp");
// large-team layout: blocks of kLargeWarps warps, one per SM
constexpr int kLargeWarps = (int)((233472 - 1024) / warp_smem_bytes<WarpSmemLarge>()) > 8
                                ? 8 : (int)((233472 - 1024) / warp_smem_bytes<WarpSmemLarge>());
static_assert(kLargeWarps >= 4, "large-team layout fits 4 warps per SM");

__device__ __forceinline__ int pair_index(int i, int j, int n) { return i * n - i * (i + 1) / 2 + (j - i - 1); }

// FFC keys order the conflicts of a query lexicographically by (t, i, j):
// key = t << kKeyShift | pair index (pairs in (i, j) order, fewer than 128).
// Per state, the colliding pairs are reduced to one code, 128 - pair index
// of the first, so the largest code names the first pair and 0 means none.
constexpr int kKeyShift = 7;
__device__ __forceinline__ unsigned pair_code(int p) { return (unsigned)(128 - p); }
__device__ __forceinline__ int code_key(int t, unsigned code) { return (t << kKeyShift) | (128 - (int)code); }

// ordered-int encoding of floats so that atomicMin on int orders like floats
__device__ __forceinline__ int f2ord(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// preparation: per-query validation, waypoint times, step count T, work shape
// ---------------------------------------------------------------------------

// ceil(|g - s|_2 / res) in IEEE double with separately rounded operations
// (no contraction), 0 when the robot does not move (Sec. IV-A3).
__device__ long long steps_from_resolution(const float *s, const float *g, int dof, float res) {
  double acc = 0.0;
  for (int k = 0; k < dof; ++k) {
    double d = __dsub_rn((double)g[k], (double)s[k]);
    acc = __dadd_rn(acc, __dmul_rn(d, d));
  }
  double dist = __dsqrt_rn(acc);
  if (dist == 0.0) return 0;
  return (long long)ceil(__ddiv_rn(dist, (double)res));
}

// Robot pairs likely to collide, for the pairs-first MV order (the mixed
// strategy Sec. III-A suggests: adjacent fixed-base manipulators first).
// Two fixed-base robots (kinematic chains) are adjacent when the distance of
// their bases is within 1.25x of either one's distance to its nearest other
// fixed base.  Sets Q.adj (bit p: pair p in (i, j) order), Q.nadj and
// Q.adjtests (sphere tests per state of the adjacent pairs).
__device__ void adjacent_pairs(const BatchDev &B, int s0, int n, QueryDev &Q) {
  float nn2[MRV_MAX_ROBOTS];
  for (int i = 0; i < n; ++i) {
    nn2[i] = INFINITY;
    const ModelDev &a = B.models[B.slot_robot_id[s0 + i]];
    if (a.kind == MRV_ROBOT_POINT) continue;
    for (int j = 0; j < n; ++j) {
      const ModelDev &b = B.models[B.slot_robot_id[s0 + j]];
      if (j == i || b.kind == MRV_ROBOT_POINT) continue;
      const float dx = a.base[3] - b.base[3], dy = a.base[7] - b.base[7], dz = a.base[11] - b.base[11];
      nn2[i] = fminf(nn2[i], dx * dx + dy * dy + dz * dz);
    }
  }
  int p = 0;
  for (int i = 0; i < n; ++i) {
    const ModelDev &a = B.models[B.slot_robot_id[s0 + i]];
    for (int j = i + 1; j < n; ++j, ++p) {
      const ModelDev &b = B.models[B.slot_robot_id[s0 + j]];
      if (a.kind == MRV_ROBOT_POINT || b.kind == MRV_ROBOT_POINT) continue;
      const float dx = a.base[3] - b.base[3], dy = a.base[7] - b.base[7], dz = a.base[11] - b.base[11];
      if (dx * dx + dy * dy + dz * dz <= 1.5625f * fmaxf(nn2[i], nn2[j])) {
        Q.adj[p >> 5] |= 1u << (p & 31);
        Q.nadj += 1;
        Q.adjtests += (long long)a.n_spheres * b.n_spheres;
      }
    }
  }
}

__global__ void k_prep(BatchDev B) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B.n_queries) return;
  uint32_t err = 0;
  QueryDev Q;
  Q.T = 0; Q.n = 0; Q.M = 0; Q.ntiles = 0; Q.split = 1; Q.spt = kWarp; Q.nslices = 0; Q.nphase = 1;
  Q.nchain = 0; Q.njoint = 0;
  Q.nchunks = 0; Q.cte = 1; Q.env = -1; Q.bits = 0; Q.rho2 = 0.f; Q.nadj = 0;
  Q.adj[0] = Q.adj[1] = Q.adj[2] = Q.adj[3] = 0u; Q.adjtests = 0;
  Q.pairtests = 0; Q.envtests = 0; Q.boxtests = 0; Q.cyltests = 0;
  const int s0 = B.q_robot_off[q], s1 = B.q_robot_off[q + 1];
  const int n = s1 - s0;
  if (n < 1 || n > MRV_MAX_ROBOTS || s0 < 0 || s1 > B.n_slots) err |= kErrRobots;
  int kind = B.forced_kind >= 0 ? B.forced_kind : (B.q_kind ? (int)B.q_kind[q] : MRV_KIND_MV);
  if (kind == MRV_KIND_FFC) Q.bits |= 1u;
  int env = B.default_env;
  if (B.q_env_id) {
    const int id = B.q_env_id[q];
    if (id == -1) env = -1;
    else if (id < kEnvIdBase || id - kEnvIdBase >= B.n_envs || !B.envs[id - kEnvIdBase].live) err |= kErrEnvId;
    else env = id - kEnvIdBase;
  }
  long long T = 0;
  int M = 0;
  bool all_point = true;
  int ms[MRV_MAX_ROBOTS];
  long long self_total = 0, self0 = 0;
  float rho2 = 0.f;
  if (!err) {
    for (int i = 0; i < n; ++i) {
      const int s = s0 + i;
      const int id = B.slot_robot_id[s];
      if (id < 0 || id >= B.n_models || !B.models[id].live) { err |= kErrRobotId; break; }
      const ModelDev &m = B.models[id];
      if (m.dof > B.wp_stride) { err |= kErrDof; break; }
      ms[i] = m.n_spheres;
      M += m.n_spheres;
      self_total += m.n_self;
      if (i == 0) self0 = m.n_self;
      rho2 = fmaxf(rho2, m.r2max);
      if (m.kind != MRV_ROBOT_POINT) {
        all_point = false;
        Q.nchain += 1;
        Q.njoint += m.dof;
      }
      const int w0 = B.slot_wp_off[s], w1 = B.slot_wp_off[s + 1];
      if (w0 < 0 || w1 <= w0 || w1 > B.n_waypoints) { err |= kErrWaypoints; break; }
      long long Ts = 0;
      if (B.seg_steps) {
        B.slot_tau[w0] = 0;
        for (int w = w0; w < w1 - 1; ++w) {
          const int st = B.seg_steps[CK(w, B.n_waypoints, SEGSTEPS, B.err)];
          if (st < 1) { err |= kErrSteps; break; }
          Ts += st;
          if (Ts > MRV_MAX_STEPS) { err |= kErrSteps; break; }
          B.slot_tau[w + 1] = (int)Ts;
        }
      } else {
        if (w1 - w0 != 2) { err |= kErrWaypoints; break; }
        const float *a = B.waypoints + (size_t)w0 * B.wp_stride;
        Ts = steps_from_resolution(a, a + B.wp_stride, m.dof, B.resolution);
        if (Ts > MRV_MAX_STEPS) err |= kErrSteps;
      }
      if (Ts > T) T = Ts;
    }
  }
  if (!err && M > MRV_MAX_QUERY_SPHERES) err |= kErrSpheres;
  if (!err && !B.seg_steps)
    for (int i = 0; i < n; ++i) {
      const int w0 = B.slot_wp_off[s0 + i];
      B.slot_tau[w0] = 0;
      B.slot_tau[w0 + 1] = (int)T;
    }
  if (err) {
    Q.bits |= 4u;
    atomicOr(B.err, err);
  } else {
    Q.T = (int)T;
    Q.n = n;
    Q.M = M;
    Q.env = env;
    Q.rho2 = rho2;
    // one lane per state (flavor A): never in the small-team default
    // instance, which keeps just the broadphase path (its code then small
    // enough for its warps to share the instruction cache); such queries
    // take the team class (the large-team one beyond 8 robots)
    const bool flavor_a = all_point && M <= kFlavorAMaxSpheres;
    if (flavor_a) Q.bits |= 2u;
    Q.bits |= (uint32_t)(flavor_a ? max(1, work_class(n, M)) : work_class(n, M)) << 3;
    const bool mv = !(Q.bits & 1u);
    const bool check_env = mv && (B.flags & MRV_CHECK_ENV);
    Q.ntiles = (int)((T + 1 + kWarp - 1) / kWarp);
    int split = flavor_a ? 1 : B.tile_split;
    if (split < 1 || split > kWarp || (split & (split - 1))) split = 4;
    Q.split = split;
    Q.spt = kWarp / split;
    Q.nslices = Q.ntiles * split;
    // hierarchical order: named by the batch, or the tuned order of early-exit
    // batches naming none (an exhaustive run visits every state in any order,
    // and two phases would only compute the link frames twice)
    const bool hier = (B.flags & MRV_HIERARCHICAL) ||
                      (B.mv_order == 1 && !(B.flags & (MRV_PAIRS_FIRST | MRV_EXHAUSTIVE)));
    Q.nphase = (check_env && hier) ? 2 : 1;
    if (mv && (B.flags & MRV_PAIRS_FIRST) && !(B.flags & MRV_EXHAUSTIVE)) {
      adjacent_pairs(B, s0, n, Q);
      if (Q.nadj > 0) Q.nphase = 2;
    }
    const int total = Q.nslices * Q.nphase;
    int cte = B.slices_per_item < 1 ? 1 : B.slices_per_item;
    const int need = (total + kMaxLevels - 1) / kMaxLevels;
    if (cte < need) cte = need;
    Q.cte = cte;
    Q.nchunks = (total + cte - 1) / cte;
    // the prioritized MV checks slot 0 alone against the obstacles and
    // itself, and only the pairs (0, j)
    const bool prio = mv && (B.flags & MRV_PRIORITY);
    long long pt = 0;
    for (int i = 0; i < (prio ? 1 : n); ++i)
      for (int j = i + 1; j < n; ++j) pt += (long long)ms[i] * ms[j];
    Q.pairtests = pt;
    long long et = 0, bt = 0, ct = 0;
    if (check_env) {
      const int Me = prio ? ms[0] : M;
      if (env >= 0) {
        et = (long long)Me * B.envs[env].n_spheres;
        bt = (long long)Me * B.envs[env].n_aabbs;
        ct = (long long)Me * B.envs[env].n_cyl;
      }
      et += prio ? self0 : self_total;
    }
    Q.envtests = et;
    Q.boxtests = bt;
    Q.cyltests = ct;
    atomicAdd(&B.stats[2], (unsigned long long)(T + 1));
    atomicAdd(&B.stats[3], (unsigned long long)((T + 1) * (pt + et + bt + ct)));
  }
  B.q[q] = Q;
  B.q_hit[q] = 0;
  B.q_best[q] = 0x7fffffff;
  B.redo_flag[q] = 0;
  B.q_states[q] = 0;
  B.q_minclr[q] = __int_as_float(f2ord(INFINITY));
  atomicAdd(&B.hist[CK((int)((Q.bits >> 3) & 3u) * (kMaxLevels + 1) + (Q.nchunks > kMaxLevels ? kMaxLevels : Q.nchunks),
                       kLevelBins, HIST, B.err)], 1);
}

// level layout, per work class: the class's queries sorted by item count
// (descending; within one item count the FFC queries, then the MV ones),
// classes in order (qbase: the queries of the classes before);
// level c holds the class's queries with more
// than c items, which are its first cnt_c sorted queries.  With h the class's
// histogram of item counts (bin kMaxLevels: that many or more) and
// S[k] = sum_{k' >= k} h[k'], the first sorted position of item count k is
// qbase + S[k + 1] and level c starts at item sum_{m <= c} S[m + 1].  One
// block of kLevelThreads threads, thread (class, k) owning bin k; both sums
// are segmented scans in shared memory.
constexpr int kLevelThreads = 1024;
static_assert(kLevelBins <= kLevelThreads, "one thread per level bin");

__device__ __forceinline__ void seg_scan(int *v, int t, int seg) {
  // inclusive prefix sums of v within segments of `seg` entries
  for (int d = 1; d < seg; d <<= 1) {
    const int add = (t < kLevelBins && t % seg >= d) ? v[t - d] : 0;
    __syncthreads();
    if (t < kLevelBins) v[t] += add;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kLevelThreads) k_levels(BatchDev B) {
  __shared__ int suf[kLevelBins], pre[kLevelBins];
  const int t = threadIdx.x, L = kMaxLevels + 1;
  const int cls = t / L, k = t - cls * L;
  // suffix sums: scan the bins in reverse order within each class
  if (t < kLevelBins) suf[cls * L + (kMaxLevels - k)] = B.hist[t];
  __syncthreads();
  seg_scan(suf, t, L);
  // S[k] of class c sits at suf[c L + kMaxLevels - k]; S[kMaxLevels + 1] = 0
  const int S1 = (t < kLevelBins && k < kMaxLevels) ? suf[cls * L + kMaxLevels - k - 1] : 0;   // S[k + 1]
  if (t < kLevelBins) pre[t] = S1;
  __syncthreads();
  seg_scan(pre, t, L);
  if (t < kLevelBins) {
    int qbase = 0;   // S[0] of each class before this one: its queries
    for (int c = 0; c < cls; ++c) qbase += suf[c * L + kMaxLevels];
    B.cursor[t] = qbase + S1;                          // FFC queries fill the bin from its start,
    B.cursor[kLevelBins + t] = qbase + S1 + B.hist[t];  // MV queries from its end
    if (k < kMaxLevels) B.level_start[CK(cls * L + k + 1, kLevelBins, LEVELS, B.err)] = pre[t];
    if (k == 0) {
      B.level_start[cls * L] = 0;
      B.counters[kCtrFirst(cls)] = qbase;
    }
    if (k == kMaxLevels - 1) B.counters[kCtrItems(cls)] = pre[t];   // the class's work items
  }
}

__global__ void k_scatter(BatchDev B) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B.n_queries) return;
  const QueryDev &Q = B.q[q];
  int c = Q.nchunks;
  if (c > kMaxLevels) c = kMaxLevels;
  // each bin holds its FFC queries first and its MV queries after them, so
  // the warps of a level run long stretches of one kind of item (one code
  // path in the instruction cache) instead of a mix
  const int bin = (int)((Q.bits >> 3) & 3u) * (kMaxLevels + 1) + c;
  const int pos = (Q.bits & 1u) ? atomicAdd(&B.cursor[bin], 1) : atomicSub(&B.cursor[kLevelBins + bin], 1) - 1;
  B.sorted[CK(pos, B.n_queries, SCATTER, B.err)] = q;
}

// ---------------------------------------------------------------------------
// per-state geometry
// ---------------------------------------------------------------------------

// configuration of slot (w0, w1) at time t: linear interpolation inside the
// waypoint segment containing t, the last waypoint once the path has ended.
__device__ __forceinline__ void interp(const BatchDev &B, int w0, int w1, int dof, int t, float *q) {
  const int last = w1 - 1;
  const int *tau = B.slot_tau;
  if (t >= tau[last]) {
    const float *a = B.waypoints + (size_t)CK(last, B.n_waypoints, WAYPOINT, B.err) * B.wp_stride;
#pragma unroll
    for (int j = 0; j < MRV_MAX_DOF; ++j)
      if (j < dof) q[j] = a[j];
    return;
  }
  int lo = w0, hi = last - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tau[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  lo = CK(lo, B.n_waypoints - 1, WAYPOINT, B.err);   // rows lo and lo + 1
  const float f = (float)(t - tau[lo]) / (float)(tau[lo + 1] - tau[lo]);
  const float *a = B.waypoints + (size_t)lo * B.wp_stride;
  const float *g = a + B.wp_stride;
#pragma unroll
  for (int j = 0; j < MRV_MAX_DOF; ++j)
    if (j < dof) q[j] = fmaf(g[j] - a[j], f, a[j]);
}

// interp from a segment hint: states only grow within a slice, so the search
// starts at the segment of the previous round (a few linear steps, then a
// binary search if still behind); *lo_out = the segment used (w1 - 1 past the
// end of the path)
__device__ __forceinline__ void interp_from(const BatchDev &B, int w0, int w1, int dof, int t, int hint, float *q,
                                            int *lo_out) {
  const int last = w1 - 1;
  const int *tau = B.slot_tau;
  if (t >= tau[last]) {
    const float *a = B.waypoints + (size_t)CK(last, B.n_waypoints, WAYPOINT, B.err) * B.wp_stride;
#pragma unroll
    for (int j = 0; j < MRV_MAX_DOF; ++j)
      if (j < dof) q[j] = a[j];
    *lo_out = last;
    return;
  }
  int lo = (hint >= w0 && hint < last && tau[hint] <= t) ? hint : w0;
  for (int s = 0; s < 4 && tau[lo + 1] <= t; ++s) ++lo;
  if (tau[lo + 1] <= t) {
    int hi = last - 1;
    ++lo;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tau[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
  }
  *lo_out = lo;
  lo = CK(lo, B.n_waypoints - 1, WAYPOINT, B.err);   // rows lo and lo + 1
  const float f = (float)(t - tau[lo]) / (float)(tau[lo + 1] - tau[lo]);
  const float *a = B.waypoints + (size_t)lo * B.wp_stride;
  const float *g = a + B.wp_stride;
#pragma unroll
  for (int j = 0; j < MRV_MAX_DOF; ++j)
    if (j < dof) q[j] = fmaf(g[j] - a[j], f, a[j]);
}

__device__ __forceinline__ void store_frame(float *X, int link, const float *R, const float *p) {
  float *o = X + link * 12;
  o[0] = R[0]; o[1] = R[1]; o[2] = R[2]; o[3] = p[0];
  o[4] = R[3]; o[5] = R[4]; o[6] = R[5]; o[7] = p[1];
  o[8] = R[6]; o[9] = R[7]; o[10] = R[8]; o[11] = p[2];
}

// SpheresFK link frames (Sec. III-A): base, then one modified-DH joint at a
// time, R' = R RotX(alpha) RotZ(theta), p' = p + a R e_x + d R' e_z, then the
// flange.  Frames are written to X[link*12] (3x4 row-major).
__device__ __noinline__ void chain_frames(const ModelDev &m, const float *q, float *X) {
  float R[9], p[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    R[3 * r + 0] = m.base[4 * r + 0];
    R[3 * r + 1] = m.base[4 * r + 1];
    R[3 * r + 2] = m.base[4 * r + 2];
    p[r] = m.base[4 * r + 3];
  }
  store_frame(X, 0, R, p);
  if (m.kind == MRV_ROBOT_POINT) {
    const float z = m.dof == 2 ? m.point_z : q[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) p[r] = fmaf(R[3 * r + 0], q[0], fmaf(R[3 * r + 1], q[1], fmaf(R[3 * r + 2], z, p[r])));
    store_frame(X, 1, R, p);
    return;
  }
#pragma unroll
  for (int k = 0; k < MRV_MAX_DOF; ++k) {
    if (k < m.dof) {
      const float ca = m.dh[k][0], sa = m.dh[k][1], a = m.dh[k][2], d = m.dh[k][3], th0 = m.th0[k];
      float s, c;
      sincosf(th0 + q[k], &s, &c);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float x = R[3 * r + 0], y = R[3 * r + 1], z = R[3 * r + 2];
        const float u = ca * y + sa * z;
        const float v = ca * z - sa * y;
        p[r] = fmaf(a, x, fmaf(d, v, p[r]));
        R[3 * r + 0] = c * x + s * u;
        R[3 * r + 1] = c * u - s * x;
        R[3 * r + 2] = v;
      }
      store_frame(X, k + 1, R, p);
    }
  }
  // flange frame dof+1 = frame dof * F
  float R2[9], p2[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2)
      R2[3 * r + c2] = R[3 * r + 0] * m.flange[c2] + R[3 * r + 1] * m.flange[4 + c2] + R[3 * r + 2] * m.flange[8 + c2];
    p2[r] = p[r] + R[3 * r + 0] * m.flange[3] + R[3 * r + 1] * m.flange[7] + R[3 * r + 2] * m.flange[11];
  }
  store_frame(X, m.dof + 1, R2, p2);
}

// One row (r = 0, 1, 2) of every link frame of a chain.  A joint mixes the
// columns of each row of the 3x4 transform but never its rows, so the rows
// evolve independently through the base, the joints and the flange, and three
// lanes can share a chain (the same arithmetic as chain_frames, row by row).
// the point (x, y, z) of a link frame's coordinates in the frame of X (3x4
// row-major, rows 16-byte aligned: three vector loads)
__device__ __forceinline__ float3 frame_apply(const float *X, float x, float y, float z) {
  const float4 *R = reinterpret_cast<const float4 *>(X);
  const float4 r0 = R[0], r1 = R[1], r2 = R[2];
  return make_float3(fmaf(r0.x, x, fmaf(r0.y, y, fmaf(r0.z, z, r0.w))),
                     fmaf(r1.x, x, fmaf(r1.y, y, fmaf(r1.z, z, r1.w))),
                     fmaf(r2.x, x, fmaf(r2.y, y, fmaf(r2.z, z, r2.w))));
}

__device__ __forceinline__ void store_row(float *X, int link, int r, float x, float y, float z, float p) {
  *reinterpret_cast<float4 *>(X + link * 12 + 4 * r) = make_float4(x, y, z, p);
}

// sin and cos of a joint angle: the angle is brought into [-pi, pi] by
// subtracting the nearest multiple of 2 pi, with 2 pi split into a float head
// and tail (Cody-Waite reduction; joint angles are a few radians, so k is
// small and the reduction exact to about 1e-7), then the hardware __sincosf,
// whose absolute error on [-pi, pi] is below 2^-21.4.  About 1e-6 rad in all,
// a hundredth of the 1e-4 m decidability margin over a 1 m arm.
__device__ __forceinline__ void joint_sincos(float x, float *s, float *c) {
  const float two_pi_hi = 6.28318548202514648f;      // float(2 pi)
  const float two_pi_lo = -1.7484556025237907e-7f;   // 2 pi - float(2 pi)
  const float k = rintf(x * 0.159154943091895336f);  // nearest multiple of 2 pi
  const float r = fmaf(-k, two_pi_lo, fmaf(-k, two_pi_hi, x));
  __sincosf(r, s, c);
}

__device__ __noinline__ void chain_row(const ModelDev &m, const float *q, float *X, int r) {
  // the model's rows are 16-byte aligned: one vector load per row and joint
  const float4 b = reinterpret_cast<const float4 *>(m.base)[r];
  float x = b.x, y = b.y, z = b.z, p = b.w;
  store_row(X, 0, r, x, y, z, p);
  if (m.kind == MRV_ROBOT_POINT) {
    const float zz = m.dof == 2 ? m.point_z : q[2];
    p = fmaf(x, q[0], fmaf(y, q[1], fmaf(z, zz, p)));
    store_row(X, 1, r, x, y, z, p);
    return;
  }
#pragma unroll
  for (int k = 0; k < MRV_MAX_DOF; ++k) {
    if (k < m.dof) {
      const float4 D = reinterpret_cast<const float4 *>(m.dh)[k];
      const float ca = D.x, sa = D.y, a = D.z, d = D.w;
      float s, c;
      joint_sincos(m.th0[k] + q[k], &s, &c);
      const float u = ca * y + sa * z;
      const float v = ca * z - sa * y;
      p = fmaf(a, x, fmaf(d, v, p));
      const float nx = c * x + s * u, ny = c * u - s * x;
      x = nx;
      y = ny;
      z = v;
      store_row(X, k + 1, r, x, y, z, p);
    }
  }
  // flange frame dof+1 = frame dof * F
  const float4 *F = reinterpret_cast<const float4 *>(m.flange);
  const float4 F0 = F[0], F1 = F[1], F2 = F[2];
  store_row(X, m.dof + 1, r, x * F0.x + y * F1.x + z * F2.x, x * F0.y + y * F1.y + z * F2.y,
            x * F0.z + y * F1.z + z * F2.z, p + x * F0.w + y * F1.w + z * F2.w);
}

// direct forms: |a - b|^2 < (ra + rb)^2, clearance |a - b| - ra - rb
__device__ __forceinline__ bool sph_hit(const float4 a, const float4 b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float rr = a.w + b.w;
  return dx * dx + dy * dy + dz * dz < rr * rr;
}

__device__ __forceinline__ float sph_clr(const float4 a, const float4 b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return sqrtf(dx * dx + dy * dy + dz * dz) - (a.w + b.w);
}

// squared distance from a point to a solid cylinder with flat caps (0
// inside): A = axis end a, radius; U = unit axis, length.  With s the axial
// coordinate and d the distance from the axis line, the nearest point of the
// solid clamps s to [0, L] and d to [0, radius].
__device__ __forceinline__ float cyl_d2(float x, float y, float z, const float4 A, const float4 U) {
  const float wx = x - A.x, wy = y - A.y, wz = z - A.z;
  const float s = fmaf(wx, U.x, fmaf(wy, U.y, wz * U.z));
  const float px = fmaf(-s, U.x, wx), py = fmaf(-s, U.y, wy), pz = fmaf(-s, U.z, wz);
  const float d2 = fmaf(px, px, fmaf(py, py, pz * pz));
  const float es = fmaxf(fmaxf(-s, s - U.w), 0.f);
  if (d2 <= A.w * A.w) return es * es;
  const float ed = sqrtf(d2) - A.w;
  return fmaf(es, es, ed * ed);
}

// squared distance from a point to a box (0 inside)
__device__ __forceinline__ float box_d2(float x, float y, float z, const float4 lo, const float4 hi) {
  const float ex = x - fminf(fmaxf(x, lo.x), hi.x);
  const float ey = y - fminf(fmaxf(y, lo.y), hi.y);
  const float ez = z - fminf(fmaxf(z, lo.z), hi.z);
  return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// expanded test value u = k_b + A . (b, r_b), A = -2 (p_a, r_a)
__device__ __forceinline__ float uval(const float4 A, const float4 b, float kb) {
  return fmaf(A.x, b.x, fmaf(A.y, b.y, fmaf(A.z, b.z, fmaf(A.w, b.w, kb))));
}

// ---------------------------------------------------------------------------
// work contexts
// ---------------------------------------------------------------------------



// state of position j of slice k (monotone in j for both packings)
__device__ __forceinline__ int slice_state(const TileCtx &C, int k, int j) {
  if (C.lin) return k * C.spt + j;
  const int b = k / C.split, p = k - b * C.split;
  return b + C.nb * (p + C.split * j);
}

// Position jj of a slice's visiting order -> its state index j.  MV in the
// rake order visits the middle of the slice first (m, m-1, m+1, m-2, ...):
// the slice's states are spread over the whole motion, and a motion between
// valid configurations collides inside it rather than at its ends, so the
// first collision is met after fewer states; the verdict does not depend on
// the order.  FFC and the linear map keep increasing states.
__device__ __forceinline__ int slot_j(const TileCtx &C, int jj, int nvalid) {
  if (C.lin) return jj;
  const int m = nvalid >> 1;   // a permutation of 0..nvalid-1 for every nvalid >= 1
  return (jj & 1) ? m - 1 - (jj >> 1) : m + (jj >> 1);
}

// number of states of slice k that lie in 0..T (its states grow with j)
__device__ __forceinline__ int slice_valid(const TileCtx &C, int k) {
  const int t0 = slice_state(C, k, 0);
  if (t0 > C.T) return 0;
  const int step = C.lin ? 1 : C.nb * C.split;
  return min(C.spt, (C.T - t0) / step + 1);
}

// ---------------------------------------------------------------------------
// flavor A: one lane per state (point robots)
// ---------------------------------------------------------------------------

// MV -> 1 if a collision was found; FFC -> smallest key (t << kKeyShift | pair) or INT_MAX
template <bool FULL, class WS>
__device__ int slice_a(const BatchDev &B, TileCtx &C, WS &S, int k, int lane, float &minclr, bool do_env,
                       bool do_pairs) {
  const int t = slice_state(C, k, lane);
  const bool valid = t <= C.T;
  float4 *PA = S.u.PA;
  if (valid) {
    for (int r = 0; r < C.n; ++r) {
      const RobotSlot &rs = S.rs[r];
      const ModelDev &m = B.models[rs.mdl];
      float q[MRV_MAX_DOF];
      interp(B, rs.w0, rs.w1, rs.dof, t, q);
      const float z = rs.dof == 2 ? m.point_z : q[2];
      for (int kk = 0; kk < rs.m; ++kk) {
        const float4 s = rs.spheres[kk];
        float lx = s.x, ly = s.y, lz = s.z;
        if (rs.links[kk] == 1) { lx += q[0]; ly += q[1]; lz += z; }
        float4 w;
        w.x = m.base[0] * lx + m.base[1] * ly + m.base[2] * lz + m.base[3];
        w.y = m.base[4] * lx + m.base[5] * ly + m.base[6] * lz + m.base[7];
        w.z = m.base[8] * lx + m.base[9] * ly + m.base[10] * lz + m.base[11];
        w.w = s.w;
        PA[CK(S.off[r] + kk, kFlavorAMaxSpheres, FLAVOR_A, C.err) * kWarp + lane] = w;
      }
    }
  }
  const int nvalid = __popc(__ballot_sync(0xffffffffu, valid));
  __syncwarp();
  if (lane == 0) {
    if (C.first_phase) C.states += nvalid;   // two-phase orders: a state counts in its first phase
    C.chains += (unsigned long long)nvalid * C.n;
    C.placed += (unsigned long long)nvalid * C.M;
  }
  __syncwarp();
  if (!C.ffc) {
    bool hit = false;
    if (valid && do_env && C.check_env) {
      for (int a = 0; a < C.env_rows; ++a) {
        const float4 pa = PA[a * kWarp + lane];
        for (int o = 0; o < C.env_ns; ++o) {
          if (C.clr) minclr = fminf(minclr, sph_clr(pa, C.env_s[o]));
          else hit |= sph_hit(pa, C.env_s[o]);
        }
        for (int o = 0; o < C.env_nb; ++o) {
          const float d2 = box_d2(pa.x, pa.y, pa.z, C.box_lo[o], C.box_hi[o]);
          if (C.clr) minclr = fminf(minclr, sqrtf(d2) - pa.w);
          else hit |= d2 < pa.w * pa.w;
        }
        for (int o = 0; o < C.env_nc; ++o) {
          const float d2 = cyl_d2(pa.x, pa.y, pa.z, __ldg(&C.cyl_a[o]), __ldg(&C.cyl_u[o]));
          if (C.clr) minclr = fminf(minclr, sqrtf(d2) - pa.w);
          else hit |= d2 < pa.w * pa.w;
        }
      }
      for (int r = 0; r < C.self_robots; ++r)
        for (int p = 0; p < S.rs[r].n_self; ++p) {
          const uint32_t sp = S.rs[r].self[p];
          const float4 x = PA[CK(S.off[r] + (int)(sp & 0xffffu), C.M, FLAVOR_A, C.err) * kWarp + lane];
          const float4 y = PA[CK(S.off[r] + (int)(sp >> 16), C.M, FLAVOR_A, C.err) * kWarp + lane];
          if (C.clr) minclr = fminf(minclr, sph_clr(x, y));
          else hit |= sph_hit(x, y);
        }
    }
    if (valid && do_pairs)
      for (int i = 0; i < C.pair_robots; ++i)
        for (int a = S.off[i]; a < S.off[i + 1]; ++a) {
          const float4 pa = PA[a * kWarp + lane];
          for (int bb = S.off[i + 1]; bb < C.M; ++bb) {
            const float4 pb = PA[bb * kWarp + lane];
            if (C.clr) minclr = fminf(minclr, sph_clr(pa, pb));
            else hit |= sph_hit(pa, pb);
          }
        }
    if (lane == 0) {
      if (do_env && C.check_env) {
        C.tests += (unsigned long long)nvalid * (unsigned long long)(C.envtests + C.boxtests + C.cyltests);
        C.btests += (unsigned long long)nvalid * (unsigned long long)C.boxtests;
        C.ctests += (unsigned long long)nvalid * (unsigned long long)C.cyltests;
      }
      if (do_pairs) C.tests += (unsigned long long)nvalid * (unsigned long long)C.pairtests;
    }
    if (C.clr) hit = minclr < 0.f;
    return __any_sync(0xffffffffu, hit) ? 1 : 0;
  }
  // FFC: first colliding pair of this lane's state, in (i, j) order
  int first = 0x7fffffff;
  if (valid)
    for (int i = 0; i < C.n && first == 0x7fffffff; ++i)
      for (int j = i + 1; j < C.n && first == 0x7fffffff; ++j) {
        bool h = false;
        for (int a = S.off[i]; a < S.off[i + 1]; ++a)
          for (int bb = S.off[j]; bb < S.off[j + 1]; ++bb) h |= sph_hit(PA[a * kWarp + lane], PA[bb * kWarp + lane]);
        if (h) first = pair_index(i, j, C.n);
      }
  if (lane == 0) C.tests += (unsigned long long)nvalid * (unsigned long long)C.pairtests;
  const unsigned m = __ballot_sync(0xffffffffu, first != 0x7fffffff);
  if (!m) return 0x7fffffff;
  const int l0 = __ffs(m) - 1;
  const int p0 = __shfl_sync(0xffffffffu, first, l0);
  return (slice_state(C, k, l0) << kKeyShift) | p0;
}

// ---------------------------------------------------------------------------
// flavor B: the warp walks the states of a slice (kinematic chains)
// ---------------------------------------------------------------------------

// decision of a row from its minimum u against threshold -k_a
__device__ __forceinline__ int decide(float m, float ka, float eps) {
  const float tau = -ka;
  return m < tau - eps ? 1 : (m < tau + eps ? 2 : 0);   // 1 hit, 2 uncertain, 0 clear
}

// Rectangle test: rows [ra, rb) of (P, shifted by sh into the column frame)
// against columns [ca, cb) of (Q, QK).  Each lane holds 4 rows (row-lane rho,
// rows base + rho + RL*r) and scans one of G = 32/RL column chunks; the row
// minima are combined over the chunks by shuffles and decided once.  Returns
// the lane's "some row collides" (callers reduce over the warp).  Rows whose
// minimum is within the rounding band are decided by the direct formula.
__device__ __noinline__ bool rect_test(const float4 *P, int ra, int rb, const float4 *Q, const float *QK, int ca,
                                       int cb, float shx, float shy, float shz, float eps, int lane) {
  const int nrows = rb - ra;
  if (nrows <= 0 || cb <= ca) return false;
  int RL = 1;
  while (RL * 4 < nrows && RL < kWarp) RL <<= 1;
  const int G = kWarp / RL;
  const int rho = lane & (RL - 1), gam = lane / RL;
  const int chunk = (cb - ca + G - 1) / G;
  const int c0 = ca + gam * chunk, c1 = min(c0 + chunk, cb);
  bool hit = false;
  for (int base = ra; base < rb; base += RL * 4) {
    float4 A[4];
    float ka[4], m[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int a = min(base + rho + RL * r, rb - 1);
      const float4 p = P[a];
      const float x = p.x + shx, y = p.y + shy, z = p.z + shz;
      A[r] = make_float4(-2.f * x, -2.f * y, -2.f * z, -2.f * p.w);
      ka[r] = fmaf(x, x, fmaf(y, y, fmaf(z, z, -p.w * p.w)));
      m[r] = INFINITY;
    }
#pragma unroll 2
    for (int c = c0; c < c1; ++c) {
      const float4 q = Q[c];
      const float qk = QK[c];
#pragma unroll
      for (int r = 0; r < 4; ++r) m[r] = fminf(m[r], uval(A[r], q, qk));
    }
    for (int o = RL; o < kWarp; o <<= 1)
#pragma unroll
      for (int r = 0; r < 4; ++r) m[r] = fminf(m[r], __shfl_xor_sync(0xffffffffu, m[r], o));
    if (gam == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int a = base + rho + RL * r;
        if (a >= rb) continue;
        int d = decide(m[r], ka[r], eps);
        if (d == 2) {   // near-tangent: the direct formula decides
          const float4 p = P[a];
          const float4 w = make_float4(p.x + shx, p.y + shy, p.z + shz, p.w);
          d = 0;
          for (int c = ca; c < cb; ++c) d |= sph_hit(w, Q[c]);
        }
        hit |= d != 0;
      }
    }
  }
  return hit;
}

// rows [ra, rb) (world = P + o) against the obstacle boxes; each lane takes
// 4 rows per round and scans every box
__device__ bool box_rows(const float4 *P, int ra, int rb, const float4 *BL, const float4 *BH, int nb, float ox,
                         float oy, float oz, int lane) {
  bool hit = false;
  for (int base = ra; base < rb; base += 4 * kWarp) {
    float4 w[4];
    float rr[4];
    bool h[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int a = min(base + lane + kWarp * r, rb - 1);
      const float4 p = P[a];
      w[r] = make_float4(p.x + ox, p.y + oy, p.z + oz, p.w);
      rr[r] = p.w * p.w;
      h[r] = false;
    }
#pragma unroll 2
    for (int o = 0; o < nb; ++o) {
      const float4 lo = BL[o], hi = BH[o];
#pragma unroll
      for (int r = 0; r < 4; ++r) h[r] |= box_d2(w[r].x, w[r].y, w[r].z, lo, hi) < rr[r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) hit |= h[r] && (base + lane + kWarp * r < rb);
  }
  return hit;
}

// MV robot-robot checks at one state: robot i's rows against every sphere of
// the robots after it
__device__ bool pairs_mv(const float4 *P, const float *K, const int *off, int n, int M, int lane, float eps,
                         int row_robots) {
  bool hit = false;
  for (int i = 0; i + 1 < n && i < row_robots; ++i)
    hit |= rect_test(P, off[i], off[i + 1], P, K, off[i + 1], M, 0.f, 0.f, 0.f, eps, lane);
  return hit;
}

// MV robot-robot checks at one state for the entries pr0..pr1-1 of the
// query's pair table
template <class WS>
__device__ bool pairs_list_mv(const float4 *P, const float *K, const WS &S, int pr0, int pr1, int lane, float eps) {
  bool hit = false;
  for (int p = pr0; p < pr1; ++p) {
    const uint32_t e = S.rp[p];
    const int i = (int)(e & 15u), j = (int)((e >> 4) & 15u);
    hit |= rect_test(P, S.off[i], S.off[i + 1], P, K, S.off[j], S.off[j + 1], 0.f, 0.f, 0.f, eps, lane);
  }
  return hit;
}

// FFC robot-robot checks at one state: code of the first colliding pair (0: none)
__device__ unsigned pairs_ffc(const float4 *P, const float *K, const int *off, int n, int lane, float eps) {
  unsigned pm = 0;
  for (int i = 0; i + 1 < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const bool h = rect_test(P, off[i], off[i + 1], P, K, off[j], off[j + 1], 0.f, 0.f, 0.f, eps, lane);
      if (__any_sync(0xffffffffu, h)) pm = max(pm, pair_code(pair_index(i, j, n)));
    }
  return pm;
}

// MV robot-obstacle checks (obstacle spheres staged in shared memory up to
// the cache size, the rest read through L1; boxes by the clamp distance) and
// self-collision pairs (rectangles of the model, or its sparse pair list)
template <class WS>
__device__ bool env_mv(const TileCtx &C, const WS &S, const float4 *P, const float *K, int lane, float cw2,
                       float eps) {
  const int M = C.env_rows;   // spheres with obstacle checks
  bool hit = false;
  if (C.env_ns) {
    const float epsw = kEpsU * (fmaxf(cw2, C.env_c2) + fmaxf(C.rho2, C.env_r2));
    hit |= rect_test(P, 0, M, C.env_s, C.env_k, 0, C.env_ns, S.ox, S.oy, S.oz, epsw, lane);
  }
  if (C.env_nb) {
    hit |= box_rows(P, 0, M, C.box_lo, C.box_hi, C.env_nb, S.ox, S.oy, S.oz, lane);
  }
  for (int a = lane; a < M && C.env_nc; a += kWarp) {   // cylinders: one row per lane
    const float4 p = P[a];
    const float x = p.x + S.ox, y = p.y + S.oy, z = p.z + S.oz, rr = p.w * p.w;
    for (int o = 0; o < C.env_nc; ++o) hit |= cyl_d2(x, y, z, __ldg(&C.cyl_a[o]), __ldg(&C.cyl_u[o])) < rr;
  }
  for (int r = 0; r < C.self_robots; ++r) {
    const int o = S.off[r];
    const int nr = S.rs[r].n_rects;
    if (nr > 0) {
      for (int k = 0; k < nr; ++k) {
        const int4 R = __ldg(&S.rs[r].rects[k]);
        CK_RANGE(R.x, R.y, S.rs[r].m, RECT, C.err);
        CK_RANGE(R.z, R.w, S.rs[r].m, RECT, C.err);
        hit |= rect_test(P, o + R.x, o + R.y, P, K, o + R.z, o + R.w, 0.f, 0.f, 0.f, eps, lane);
      }
    } else {
      // sparse pairs (sorted): consecutive lanes take consecutive pairs, so
      // a warp's first spheres mostly coincide and its second spheres are
      // adjacent (no bank conflicts); four pairs per lane per round
      const int ns = S.rs[r].n_self;
      const uint32_t *sp = S.rs[r].self;
      const float4 *Pr = P + o;
      for (int p0 = 0; p0 < ns; p0 += 4 * kWarp) {
        uint32_t e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = p0 + lane + kWarp * u;
          e[u] = p < ns ? __ldg(&sp[p]) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (p0 + lane + kWarp * u < ns)
            hit |= sph_hit(Pr[CK((int)(e[u] & 0xffffu), S.rs[r].m, SELF_PAIR, C.err)],
                           Pr[CK((int)(e[u] >> 16), S.rs[r].m, SELF_PAIR, C.err)]);
      }
    }
  }
  return hit;
}

// ---------------------------------------------------------------------------
// frame-level broadphase (default for kinematic chains)
// ---------------------------------------------------------------------------
// Every frame of every robot carries a bounding sphere of its spheres
// (enlarged so that an FP32 separation test is conservative).  Sphere tests
// run only for frame pairs (and frame / obstacle pairs) whose bounding spheres
// overlap; all others cannot hold a collision.  Verdicts are those of the
// full test.

// bounding spheres of every (robot, frame) at the state whose frames sit in
// FK slot jj of xf
template <class WS>
__device__ void link_spheres(const TileCtx &C, WS &S, const float *xf, int jj, int lane) {
  const int n = C.n, nef = C.nef;
  for (int i = lane; i < nef; i += kWarp) {
    const int k = CK((int)S.ef[i], WS::kRobots * kMaxLinks, FRAME_SLOT, C.err);
    const int r = k / kMaxLinks, l = k - r * kMaxLinks;
    const float4 bs = reinterpret_cast<const float4 *>(S.rs[r].md->link_bs)[l];
    const float *X = xf + (CK(jj * n + r, WS::kChains, CHAIN, C.err) * kMaxLinks + l) * 12;
    const float3 w = frame_apply(X, bs.x, bs.y, bs.z);
    S.BS[k] = make_float4(w.x - S.ox, w.y - S.oy, w.z - S.oz, bs.w);
  }
}

// robot-robot checks: MV -> 1 on a collision; FFC -> code of the first
// colliding pair (0: none).  Lane k owns the bounding sphere of (robot i, frame u) and scans the
// frame spheres of every later robot (broadcast reads); where two overlap
// the lane tests their spheres itself (overlaps are rare).
template <class WS>
__device__ unsigned pairs_broad(const TileCtx &C, const WS &S, const float4 *P, int lane, bool ffc,
                                unsigned long long &ntests) {
  unsigned pm = 0;
  const int nk = C.n * kMaxLinks;
  for (int k0 = 0; k0 < nk; k0 += kWarp) {
    const int k = k0 + lane;
    const int i = k / kMaxLinks, u = k - i * kMaxLinks;   // constant divisor
    const float4 bu = k < nk ? S.BS[k] : make_float4(0.f, 0.f, 0.f, -1.f);
    if (bu.w >= 0.f && i < C.pair_robots) {
      const int a0 = S.off[i] + S.rs[i].ls[u], a1 = CK(S.off[i] + S.rs[i].ls[u + 1], C.M + 1, SPHERE, C.err);
      for (int k2 = (i + 1) * kMaxLinks; k2 < nk; ++k2) {
        const float4 bv = S.BS[k2];
        if (bv.w < 0.f) continue;
        ntests += 1;
        if (!sph_hit(bu, bv)) continue;
        const int j = k2 / kMaxLinks, v = k2 - j * kMaxLinks;
        const int b0 = S.off[j] + S.rs[j].ls[v], b1 = CK(S.off[j] + S.rs[j].ls[v + 1], C.M + 1, SPHERE, C.err);
        bool h = false;
        for (int a = a0; a < a1 && !h; ++a) {
          const float4 pa = P[a];
          for (int b = b0; b < b1; ++b) h |= sph_hit(pa, P[b]);
          ntests += (unsigned long long)(b1 - b0);
        }
        if (h) pm = ffc ? max(pm, pair_code(pair_index(i, j, C.n))) : 1u;
      }
    }
  }
  return pm;
}

// robot-obstacle and self checks (MV with the environment).  Lane k owns
// the bounding sphere of (robot r, frame l) and scans the obstacle spheres and
// boxes (broadcast reads); overlaps are resolved sphere by sphere in the lane.
template <class WS>
__device__ bool env_broad(const TileCtx &C, const WS &S, const float4 *P, int lane, unsigned long long &ntests,
                          unsigned long long &nbox, unsigned long long &ncyl) {
  bool hit = false;
  const int nk = C.self_robots * kMaxLinks;   // frames of the robots with obstacle checks
  for (int k0 = 0; k0 < nk; k0 += kWarp) {
    const int k = k0 + lane;
    const float4 bl = k < nk ? S.BS[k] : make_float4(0.f, 0.f, 0.f, -1.f);
    if (bl.w < 0.f) continue;
    const int r = k / kMaxLinks, l = k - r * kMaxLinks;
    const int a0 = S.off[r] + S.rs[r].ls[l], a1 = CK(S.off[r] + S.rs[r].ls[l + 1], C.M + 1, SPHERE, C.err);
    const float4 bw = make_float4(bl.x + S.ox, bl.y + S.oy, bl.z + S.oz, bl.w);
    for (int e = 0; e < C.env_ns; ++e) {
      const float4 es = __ldg(&C.env_s[e]);
      ntests += 1;
      if (!sph_hit(bw, es)) continue;
      for (int a = a0; a < a1; ++a) {
        const float4 p = P[a];
        hit |= sph_hit(make_float4(p.x + S.ox, p.y + S.oy, p.z + S.oz, p.w), es);
        ntests += 1;
      }
    }
    const float rr = bw.w * bw.w;
    for (int b = 0; b < C.env_nb; ++b) {
      const float4 lo = __ldg(&C.box_lo[b]);
      const float4 hi = __ldg(&C.box_hi[b]);
      ntests += 1;
      nbox += 1;
      if (!(box_d2(bw.x, bw.y, bw.z, lo, hi) < rr)) continue;
      for (int a = a0; a < a1; ++a) {
        const float4 p = P[a];
        hit |= box_d2(p.x + S.ox, p.y + S.oy, p.z + S.oz, lo, hi) < p.w * p.w;
        ntests += 1;
        nbox += 1;
      }
    }
    for (int y = 0; y < C.env_nc; ++y) {
      const float4 A = __ldg(&C.cyl_a[y]), U = __ldg(&C.cyl_u[y]);
      ntests += 1;
      ncyl += 1;
      if (!(cyl_d2(bw.x, bw.y, bw.z, A, U) < rr)) continue;
      for (int a = a0; a < a1; ++a) {
        const float4 p = P[a];
        hit |= cyl_d2(p.x + S.ox, p.y + S.oy, p.z + S.oz, A, U) < p.w * p.w;
        ntests += 1;
        ncyl += 1;
      }
    }
  }
  if (!C.exhaustive && __any_sync(0xffffffffu, hit)) return true;
  // self pairs, grouped by frame pair: lanes test the groups' bounding
  // spheres, then the warp walks the overlapping groups' pairs together
  for (int r = 0; r < C.self_robots; ++r) {
    const ModelDev &md = *S.rs[r].md;
    const int o = S.off[r];
    const int ng = S.rs[r].n_groups;
    for (int g0 = 0; g0 < ng; g0 += kWarp) {
      const int g = g0 + lane;
      int4 G = make_int4(0, 0, 0, 0);
      bool ov = false;
      if (g < ng) {
        G = __ldg(&md.self_groups[g]);
        ov = sph_hit(S.BS[r * kMaxLinks + CK(G.x, S.rs[r].n_links, SELF_GROUP, C.err)],
                     S.BS[r * kMaxLinks + CK(G.y, S.rs[r].n_links, SELF_GROUP, C.err)]);
        ntests += 1;
      }
      unsigned m = __ballot_sync(0xffffffffu, ov);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int gs = __shfl_sync(0xffffffffu, G.z, src), gc = __shfl_sync(0xffffffffu, G.w, src);
        for (int p = lane; p < gc; p += kWarp) {
          const uint32_t e = __ldg(&md.self_pairs[CK(gs + p, (S.rs[r].n_self + 3) & ~3, SELF_PAIR, C.err)]);
          hit |= sph_hit(P[o + CK((int)(e & 0xffffu), S.rs[r].m, SELF_PAIR, C.err)],
                         P[o + CK((int)(e >> 16), S.rs[r].m, SELF_PAIR, C.err)]);
          ntests += 1;
        }
      }
    }
  }
  return hit;
}

// --- candidate-list broadphase with lazy sphere placement -------------------
//
// Per state: the frames' bounding spheres are tested against the obstacles,
// each other (self-pair groups) and the other robots' frames; overlaps go to
// per-warp candidate lists and mark the frames involved.  Only those frames'
// spheres are placed, and the exact tests of the lists are spread over the
// lanes as one flat index space (candidate x sphere).  A list that overflows
// sends its phase to the in-lane path with every sphere placed.

struct BroadAcc {            // per-lane statistics of a slice
  uint32_t tests, boxes, placed, cyls;
};

__device__ __forceinline__ void push_cand(uint32_t *list, int32_t *count, int32_t *overflow, uint32_t v) {
  const int i = atomicAdd(count, 1);
  if (i < kCand) list[i] = v;
  else *overflow = 1;
}

// frame slot k with an obstacle index e; indices past 24 bits go to the
// in-lane path through the overflow flag
__device__ __forceinline__ void push_obst(uint32_t *list, int32_t *count, int32_t *overflow, int k, int e) {
  if (e > 0xffffff) *overflow = 1;
  else push_cand(list, count, overflow, ((uint32_t)k << 24) | (uint32_t)e);
}

template <class CL>
__device__ __forceinline__ void need_frame(CL &cl, int k) { atomicOr(&cl.need[k >> 5], 1u << (k & 31)); }

// Exclusive prefix of the per-item test counts c (lane i0 + lane holds item
// i0 + lane's) into pf, called for i0 = 0, 32, ...; returns the new base.
__device__ __forceinline__ int scan_chunk(int32_t *pf, int i, int n, int c, int base, int lane) {
  int x = c;
#pragma unroll
  for (int d = 1; d < kWarp; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (i < n) pf[i] = base + x - c;
  return base + __shfl_sync(0xffffffffu, x, kWarp - 1);
}

template <class WS>
__device__ __forceinline__ int frame_count(const WS &S, int k) {
  const int r = k / kMaxLinks, l = k - r * kMaxLinks;
  return S.rs[r].ls[l + 1] - S.rs[r].ls[l];
}

template <class WS>
__device__ __forceinline__ int frame_first(const WS &S, int k) {
  const int r = k / kMaxLinks, l = k - r * kMaxLinks;
  return S.off[r] + S.rs[r].ls[l];
}

// prefix of spheres-per-frame over a list of frame-slot << 24 entries
template <class CL, class WS>
__device__ int scan_frames(CL &cl, const uint32_t *list, int n, const WS &S, int lane) {
  int base = 0;
  for (int i0 = 0; i0 < n; i0 += kWarp) {
    const int i = i0 + lane;
    const int c = i < n ? frame_count(S, (int)(list[i] >> 24)) : 0;
    base = scan_chunk(cl.pf, i, n, c, base, lane);
  }
  if (lane == 0) cl.pf[n] = base;
  __syncwarp();
  return base;
}

// places the spheres of the frames marked in cl.need and not placed yet
template <class WS>
__device__ void place_needed(const TileCtx &C, WS &S, const float *xf, int jj, int lane, BroadAcc &acc) {
  auto &cl = S.u.b.cl;
  constexpr int NW = WS::Cl::kWords;
  uint32_t any = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) any |= cl.need[w] & ~cl.placed[w];
  if (!any) return;
  float4 *P = S.u.b.P;
  const int n = C.n;
  for (int r = 0; r < n; ++r) {
    const int k0 = r * kMaxLinks, wd = k0 >> 5, sh = k0 & 31;
    const uint32_t lo = cl.need[wd] & ~cl.placed[wd];
    const uint32_t hi = wd + 1 < NW ? cl.need[wd + 1] & ~cl.placed[wd + 1] : 0u;
    const uint32_t mr = (uint32_t)((((unsigned long long)hi << 32) | lo) >> sh) & ((1u << kMaxLinks) - 1u);
    if (!mr) continue;
    const float *Xr = xf + CK(jj * n + r, WS::kChains, CHAIN, C.err) * (kMaxLinks * 12);
    const float4 *sph = S.rs[r].spheres;
    const int32_t *lnk = S.rs[r].links;
    const int a0 = S.off[r];
    // spheres are sorted by frame: walk from the first to the last frame to place
    const int s0 = S.rs[r].ls[__ffs(mr) - 1], s1 = S.rs[r].ls[32 - __clz(mr)];
    for (int kk = s0 + lane; kk < s1; kk += kWarp) {
      // both loads issued together (the sphere is read even where its frame
      // is not needed)
      const int l = CK(__ldg(&lnk[kk]), S.rs[r].n_links, LINK, C.err);
      const float4 sp = __ldg(&sph[kk]);
      if (!((mr >> l) & 1u)) continue;
      const float3 w = frame_apply(Xr + l * 12, sp.x, sp.y, sp.z);
      P[CK(a0 + kk, C.M, SPHERE, C.err)] = make_float4(w.x - S.ox, w.y - S.oy, w.z - S.oz, sp.w);
      acc.placed += 1;
    }
  }
  __syncwarp();
  if (lane == 0) {
#pragma unroll
    for (int w = 0; w < NW; ++w) cl.placed[w] |= cl.need[w];
  }
  __syncwarp();
}

template <class CL>
__device__ __forceinline__ void need_all(CL &cl, int lane) {
  if (lane == 0)
#pragma unroll
    for (int w = 0; w < CL::kWords; ++w) cl.need[w] = 0xffffffffu;
  __syncwarp();
}

// last item i of a prefix list with pf[i] <= f (f < pf[n])
__device__ __forceinline__ int list_find(const int32_t *pf, int n, int f) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pf[mid] <= f) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Exact tests of a frame x obstacle list (cl.pf holds its sphere prefix):
// lane l takes a contiguous run of the flat (candidate, sphere) range, so a
// candidate's data stays in registers over its spheres.
template <int KIND, class WS>   // KIND 0: obstacle spheres, 1: boxes, 2: cylinders
__device__ bool resolve_obstacles(const TileCtx &C, const WS &S, const uint32_t *list, int n, int tot,
                                  int lane, BroadAcc &acc) {
  const auto &cl = S.u.b.cl;
  const float4 *P = S.u.b.P;
  const int per = (tot + kWarp - 1) / kWarp;
  int f = lane * per;
  const int fe = min(f + per, tot);
  bool hit = false;
  if (f < fe) {
    acc.tests += (uint32_t)(fe - f);
    if (KIND == 1) acc.boxes += (uint32_t)(fe - f);
    if (KIND == 2) acc.cyls += (uint32_t)(fe - f);
    const float ox = S.ox, oy = S.oy, oz = S.oz;
    for (int it = list_find(cl.pf, n, f); f < fe; ++it) {
      const uint32_t v = list[CK(it, kCand, CAND, C.err)];
      const int o = CK((int)(v & 0xffffffu), KIND == 0 ? C.env_ns : (KIND == 1 ? C.env_nb : C.env_nc),
                       CAND, C.err);
      const int ge = min(fe, cl.pf[it + 1]);
      const int k = CK((int)(v >> 24), WS::kRobots * kMaxLinks, CAND, C.err);
      CK_RANGE(frame_first(S, k) + (f - cl.pf[it]), frame_first(S, k) + (ge - cl.pf[it]), C.M, SPHERE, C.err);
      const float4 *Pk = P + frame_first(S, k) - cl.pf[it];
      if (KIND == 0) {
        const float4 es = __ldg(&C.env_s[o]);
#pragma unroll 4
        for (; f < ge; ++f) {
          const float4 p = Pk[f];
          hit |= sph_hit(make_float4(p.x + ox, p.y + oy, p.z + oz, p.w), es);
        }
      } else if (KIND == 2) {
        const float4 A = __ldg(&C.cyl_a[o]), U = __ldg(&C.cyl_u[o]);
        for (; f < ge; ++f) {
          const float4 p = Pk[f];
          hit |= cyl_d2(p.x + ox, p.y + oy, p.z + oz, A, U) < p.w * p.w;
        }
      } else {
        const float4 lo = __ldg(&C.box_lo[o]);
        const float4 hi = __ldg(&C.box_hi[o]);
#pragma unroll 4
        for (; f < ge; ++f) {
          const float4 p = Pk[f];
          hit |= box_d2(p.x + ox, p.y + oy, p.z + oz, lo, hi) < p.w * p.w;
        }
      }
    }
  }
  return hit;
}

// Resolves the self-pair groups in the candidate list (blocks: lane = one
// row sphere of a group's block; pair lists: contiguous runs per lane), after
// placing the frames they need; returns this lane's hit and empties the list.
// The large-team instance calls it once per batch of groups; the team
// instance keeps the same steps inline in broad_state (as a call they
// measured about 3% slower there).
template <class WS>
__device__ bool resolve_self_list(const TileCtx &C, WS &S, const float *xf, int jj, int lane, BroadAcc &acc) {
  auto &cl = S.u.b.cl;
  const float4 *P = S.u.b.P;
  bool hit = false;
  if (!cl.ns) return false;
  if (C.self_blk) {
    // self pairs as blocks: lane = one row sphere of an overlapping
    // group's block, tested against the columns its mask lists (lanes of
    // one block read the same column spheres)
    place_needed(C, S, xf, jj, lane, acc);
    const int ns = cl.ns;
    int base = 0;
    for (int i0 = 0; i0 < ns; i0 += kWarp) {
      const int i = i0 + lane;
      int c = 0;
      if (i < ns) {
        const uint32_t v = cl.sc[i];
        const int r = CK((int)(v >> 16), C.n, SELF_BLOCK, C.err);
        const int4 Bk = __ldg(&S.rs[r].md->self_blocks[CK((int)(v & 0xffffu), S.rs[r].n_groups, SELF_BLOCK, C.err)]);
        const int o = S.off[r];
        c = Bk.z & 0xffff;
        CK_RANGE(o + Bk.x, o + Bk.x + c, min(C.M, 1024), SELF_BLOCK, C.err);
        CK_RANGE(o + Bk.y, o + Bk.y + ((Bk.z >> 16) & 0xff), min(C.M, 1024), SELF_BLOCK, C.err);
        CK_RANGE(Bk.w, Bk.w + c, min(S.rs[r].md->n_masks, 65536), SELF_MASK, C.err);
        cl.sc[i] = (uint32_t)(o + Bk.x) | ((uint32_t)(o + Bk.y) << 10) | ((uint32_t)r << 20);
        cl.scn[i] = (uint16_t)Bk.w;
        cl.sck[i] = (uint8_t)(r * kMaxLinks + CK((Bk.z >> 24) & 15, S.rs[r].n_links, SELF_BLOCK, C.err));
      }
      base = scan_chunk(cl.pf, i, ns, c, base, lane);
    }
    if (lane == 0) cl.pf[ns] = base;
    __syncwarp();
    int it = 0;
    uint32_t nt = 0;
    for (int f = lane; f < base; f += kWarp) {
      while (cl.pf[it + 1] <= f) ++it;
      const uint32_t v = cl.sc[it];
      const int row = f - cl.pf[it];
      const float4 pa = P[(int)(v & 1023u) + row];
      // a row sphere clear of the column frame's bounding sphere is clear
      // of every column sphere
      nt += 1;
      if (!sph_hit(pa, S.BS[cl.sck[it]])) continue;
      const float4 *Pc = P + ((v >> 10) & 1023u);
      uint32_t mk = __ldg(&S.rs[v >> 20].masks[cl.scn[it] + row]);
      nt += (uint32_t)__popc(mk);
      while (mk) {
        const int c = __ffs(mk) - 1;
        mk &= mk - 1;
        hit |= sph_hit(pa, Pc[CK((int)((v >> 10) & 1023u) + c, C.M, SELF_MASK, C.err) - (int)((v >> 10) & 1023u)]);
      }
    }
    acc.tests += nt;
    __syncwarp();
  } else {
    // self pairs from the pair list, one contiguous run per lane
    place_needed(C, S, xf, jj, lane, acc);
    const int ns = cl.ns;
    int base = 0;
    for (int i0 = 0; i0 < ns; i0 += kWarp) {
      const int i = i0 + lane;
      int c = 0;
      if (i < ns) c = cl.scn[i];
      base = scan_chunk(cl.pf, i, ns, c, base, lane);
    }
    if (lane == 0) cl.pf[ns] = base;
    __syncwarp();
    const int per = (base + kWarp - 1) / kWarp;
    int f = lane * per;
    const int fe = min(f + per, base);
    if (f < fe) {
      acc.tests += (uint32_t)(fe - f);
      for (int it = list_find(cl.pf, ns, f); f < fe; ++it) {
        const uint32_t v = cl.sc[it];
        const int r = (int)(v >> 16);
        const int ge = min(fe, cl.pf[it + 1]);
        const uint32_t *pr = S.rs[r].self + (int)(v & 0xffffu) - cl.pf[it];
        const float4 *Pr = P + S.off[r];
        CK_RANGE((int)(v & 0xffffu) + (f - cl.pf[it]), (int)(v & 0xffffu) + (ge - cl.pf[it]),
                 (S.rs[r].n_self + 3) & ~3, SELF_PAIR, C.err);
#pragma unroll 4
        for (; f < ge; ++f) {
          const uint32_t e = __ldg(&pr[f]);
          hit |= sph_hit(Pr[CK((int)(e & 0xffffu), S.rs[r].m, SELF_PAIR, C.err)],
                         Pr[CK((int)(e >> 16), S.rs[r].m, SELF_PAIR, C.err)]);
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0) cl.ns = 0;
  __syncwarp();
  return hit;
}

__device__ EnvDev g_no_env;   // zero: no obstacles, an empty grid

// One state of the broadphase path: MV -> 1 on a collision, FFC -> the
// code of the first colliding robot pair (0: none).  MV checks the obstacles, then the self
// pairs, then the other robots, with a warp vote after each (all three
// belong to one state, so the verdict is the same in any order; the env and
// self checks still come before the robot-robot ones, as in Alg. 1).
// kRedoState: the state needs a path only the full instance has (a
// candidate list overflowed, or self pairs without blocks); the default
// instance then hands the whole query over (FULL = false only)
constexpr unsigned kRedoState = 0xffffffffu;
constexpr int kSliceRedo = -2;   // slice result: hand the query over
// only the small-team default instance hands queries over (the one whose
// code must stay small: it runs the bulk of mixed batches); the team and
// large-team instances keep the in-lane fallbacks, since their 8- and
// 16-arm queries overflow the lists often
template <bool FULL, class WS>
__host__ __device__ constexpr bool hands_over() { return !FULL && WS::kClass == 0; }

template <bool FULL, class WS>
__device__ unsigned broad_state(TileCtx &C, WS &S, const float *xf, int jj, int lane, bool need_env,
                                bool do_pairs, BroadAcc &acc) {
  auto &cl = S.u.b.cl;
  const float4 *P = S.u.b.P;
  const int n = C.n;
  const int nke = C.nef_env;   // frames with obstacle checks: entries [0, nke) of ef
  const bool exhaustive = C.exhaustive != 0, ffc = C.ffc != 0;
  if (lane == 0) {
    cl.np = cl.ne = cl.nb = cl.ns = cl.overflow = cl.ny = 0;
#pragma unroll
    for (int w = 0; w < WS::Cl::kWords; ++w) cl.need[w] = cl.placed[w] = 0u;
  }
  __syncwarp();
  bool hit = false;
  if (need_env) {
    const int env_ns = C.env_ns, env_nb = C.env_nb;
    const float4 *env_s = C.env_s, *box_lo = C.box_lo, *box_hi = C.box_hi;
    const float ox = S.ox, oy = S.oy, oz = S.oz;
    // lane per frame: the obstacles listed in the grid cell of its center;
    // a frame larger than the grid's radius, or any frame when the
    // environment has no grid, scans every obstacle
    // (no environment: an empty one, whose frames find no grid cell)
    const EnvDev *Ep = C.env ? C.env : &g_no_env;
    const float gR = Ep->g_R;
    const float glx = Ep->g_lo[0], gly = Ep->g_lo[1], glz = Ep->g_lo[2], gih = Ep->g_inv_h;
    const int gdx = Ep->g_dims[0], gdy = Ep->g_dims[1], gdz = Ep->g_dims[2];
    {
      for (int i = lane; i < nke; i += kWarp) {
        const int k = S.ef[i];
        const float4 bl = S.BS[k];
        const float4 bw = make_float4(bl.x + ox, bl.y + oy, bl.z + oz, bl.w);
        int i0 = 0, is = 0, ib = 0, i1 = 0;   // spheres [i0, is), boxes [is, ib), cylinders [ib, i1)
        bool full = false;
        if (bw.w <= gR) {
          const float fx = (bw.x - glx) * gih, fy = (bw.y - gly) * gih, fz = (bw.z - glz) * gih;
          if (fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)gdx && fy < (float)gdy && fz < (float)gdz) {
            const int c = CK(((int)fz * gdy + (int)fy) * gdx + (int)fx, gdx * gdy * gdz, GRID_CELL, C.err);
            i0 = __ldg(&Ep->g_off[c]);
            i1 = __ldg(&Ep->g_off[c + 1]);
            const uint32_t cnt = __ldg(&Ep->g_cnt[c]);
            is = i0 + (int)(cnt & 0xffffu);
            ib = is + (int)(cnt >> 16);
          }
        } else {
          full = true;
        }
        bool nd = false;
        if (!full) {
          acc.tests += (uint32_t)(i1 - i0);
          acc.boxes += (uint32_t)(ib - is);
          acc.cyls += (uint32_t)(i1 - ib);
          CK_RANGE(i0, i1, Ep->g_nitems, GRID_ITEM, C.err);
          for (int i = i0; i < is; ++i) {
            const int e = CK((int)__ldg(&Ep->g_items[i]), env_ns, OBST_SPHERE, C.err);
            const float4 es = __ldg(&env_s[e]);
            if (sph_hit(bw, es)) {
              push_obst(cl.ec, &cl.ne, &cl.overflow, k, e);
              nd = true;
            }
          }
          const float rr = bw.w * bw.w;
          for (int i = is; i < ib; ++i) {
            const int b = CK((int)__ldg(&Ep->g_items[i]), env_nb, OBST_BOX, C.err);
            const float4 lo = __ldg(&box_lo[b]);
            const float4 hi = __ldg(&box_hi[b]);
            if (box_d2(bw.x, bw.y, bw.z, lo, hi) < rr) {
              push_obst(cl.bc, &cl.nb, &cl.overflow, k, b);
              nd = true;
            }
          }
          for (int i = ib; i < i1; ++i) {
            const int y = CK((int)__ldg(&Ep->g_items[i]), C.env_nc, OBST_CYL, C.err);
            if (cyl_d2(bw.x, bw.y, bw.z, __ldg(&C.cyl_a[y]), __ldg(&C.cyl_u[y])) < rr) {
              push_obst(cl.yc, &cl.ny, &cl.overflow, k, y);
              nd = true;
            }
          }
        } else {
          acc.tests += (uint32_t)(env_ns + env_nb + C.env_nc);
          acc.boxes += (uint32_t)env_nb;
          acc.cyls += (uint32_t)C.env_nc;
          for (int e = 0; e < env_ns; ++e) {
            const float4 es = __ldg(&env_s[e]);
            if (sph_hit(bw, es)) {
              push_obst(cl.ec, &cl.ne, &cl.overflow, k, e);
              nd = true;
            }
          }
          const float rr = bw.w * bw.w;
          for (int b = 0; b < env_nb; ++b) {
            const float4 lo = __ldg(&box_lo[b]);
            const float4 hi = __ldg(&box_hi[b]);
            if (box_d2(bw.x, bw.y, bw.z, lo, hi) < rr) {
              push_obst(cl.bc, &cl.nb, &cl.overflow, k, b);
              nd = true;
            }
          }
          for (int y = 0; y < C.env_nc; ++y)
            if (cyl_d2(bw.x, bw.y, bw.z, __ldg(&C.cyl_a[y]), __ldg(&C.cyl_u[y])) < rr) {
              push_obst(cl.yc, &cl.ny, &cl.overflow, k, y);
              nd = true;
            }
        }
        if (nd) need_frame(cl, k);
      }
    }
    __syncwarp();
    if (hands_over<FULL, WS>() && cl.overflow) return kRedoState;
    if (!hands_over<FULL, WS>() && cl.overflow) {   // too many candidates: resolve env and self in the lanes
      need_all(cl, lane);
      place_needed(C, S, xf, jj, lane, acc);
      unsigned long long t = 0, bx = 0, cy = 0;
      hit = env_broad(C, S, P, lane, t, bx, cy);
      acc.tests += (uint32_t)t;
      acc.boxes += (uint32_t)bx;
      acc.cyls += (uint32_t)cy;
      if (__any_sync(0xffffffffu, hit) && !exhaustive) return 1u;
    } else {
      if (cl.ne | cl.nb | cl.ny) {
        place_needed(C, S, xf, jj, lane, acc);
        const int ne = cl.ne, nbx = cl.nb, ny = cl.ny;
        if (ne) {
          const int tot = scan_frames(cl, cl.ec, ne, S, lane);
          hit |= resolve_obstacles<0>(C, S, cl.ec, ne, tot, lane, acc);
          __syncwarp();
        }
        if (nbx) {
          const int tot = scan_frames(cl, cl.bc, nbx, S, lane);
          hit |= resolve_obstacles<1>(C, S, cl.bc, nbx, tot, lane, acc);
          __syncwarp();
        }
        if (ny) {
          const int tot = scan_frames(cl, cl.yc, ny, S, lane);
          hit |= resolve_obstacles<2>(C, S, cl.yc, ny, tot, lane, acc);
          __syncwarp();
        }
        if (__any_sync(0xffffffffu, hit) && !exhaustive) return 1u;
      }
      // self-pair groups by their frames' bounding spheres
      if constexpr (WS::kLarge) {
        // large teams: 32 groups at a time, the overlapping ones appended to
        // the list in order, and the list resolved (with a vote) whenever the
        // next 32 might not fit, so it never overflows (16 arms: about 100 of
        // 432 groups overlap at a state)
        for (int r = 0; r < C.self_robots; ++r) {
          const int4 *groups = S.rs[r].md->self_groups;
          const int ng = S.rs[r].n_groups;
          for (int g0 = 0; g0 < ng; g0 += kWarp) {
            const int g = g0 + lane;
            int4 G = make_int4(0, 0, 0, 0);
            bool ov = false;
            if (g < ng) {
              G = __ldg(&groups[g]);
              acc.tests += 1;
              ov = sph_hit(S.BS[r * kMaxLinks + CK(G.x, S.rs[r].n_links, SELF_GROUP, C.err)],
                           S.BS[r * kMaxLinks + CK(G.y, S.rs[r].n_links, SELF_GROUP, C.err)]);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ov);
            if (!m) continue;
            if (cl.ns + __popc(m) > kCand) {
              hit |= resolve_self_list(C, S, xf, jj, lane, acc);
              if (__any_sync(0xffffffffu, hit) && !exhaustive) return 1u;
            }
            if (ov) {
              const int i = CK(cl.ns + __popc(m & ((1u << lane) - 1u)), kCand, CAND, C.err);
              // blocks: robot << 16 | group; pair list: robot << 16 | first pair
              cl.sc[i] = ((uint32_t)r << 16) | (uint32_t)(C.self_blk ? g : G.z);
              cl.scn[i] = (uint16_t)G.w;
              need_frame(cl, r * kMaxLinks + G.x);
              need_frame(cl, r * kMaxLinks + G.y);
            }
            __syncwarp();
            if (lane == 0) cl.ns += __popc(m);
            __syncwarp();
          }
        }
        hit |= resolve_self_list(C, S, xf, jj, lane, acc);
      } else {
        // team layout: one pass (about 25 of the 4-arm cage's 108 groups
        // overlap); an overflowing list sends env and self to the lanes
        for (int r = 0; r < C.self_robots; ++r) {
          const int4 *groups = S.rs[r].md->self_groups;
          const int ng = S.rs[r].n_groups;
          for (int g = lane; g < ng; g += kWarp) {
            const int4 G = __ldg(&groups[g]);
            acc.tests += 1;
            if (sph_hit(S.BS[r * kMaxLinks + CK(G.x, S.rs[r].n_links, SELF_GROUP, C.err)],
                        S.BS[r * kMaxLinks + CK(G.y, S.rs[r].n_links, SELF_GROUP, C.err)])) {
              const int i = atomicAdd(&cl.ns, 1);
              if (i < kCand) {
                // blocks: robot << 16 | group; pair list: robot << 16 | first pair
                cl.sc[i] = ((uint32_t)r << 16) | (uint32_t)(C.self_blk ? g : G.z);
                cl.scn[i] = (uint16_t)G.w;
              } else {
                cl.overflow = 1;
              }
              need_frame(cl, r * kMaxLinks + G.x);
              need_frame(cl, r * kMaxLinks + G.y);
            }
          }
        }
        __syncwarp();
        if (hands_over<FULL, WS>() && (cl.overflow || (cl.ns && !C.self_blk))) return kRedoState;
        if (!hands_over<FULL, WS>() && cl.overflow) {
          need_all(cl, lane);
          place_needed(C, S, xf, jj, lane, acc);
          unsigned long long t = 0, bx = 0, cy = 0;
          hit |= env_broad(C, S, P, lane, t, bx, cy);
          acc.tests += (uint32_t)t;
          acc.boxes += (uint32_t)bx;
          acc.cyls += (uint32_t)cy;
        } else if (cl.ns && C.self_blk) {
          // self pairs as blocks: lane = one row sphere of an overlapping
          // group's block, tested against the columns its mask lists (lanes of
          // one block read the same column spheres)
          place_needed(C, S, xf, jj, lane, acc);
          const int ns = cl.ns;
          int base = 0;
          for (int i0 = 0; i0 < ns; i0 += kWarp) {
            const int i = i0 + lane;
            int c = 0;
            if (i < ns) {
              const uint32_t v = cl.sc[i];
              const int r = CK((int)(v >> 16), C.n, SELF_BLOCK, C.err);
              const int4 Bk = __ldg(&S.rs[r].md->self_blocks[CK((int)(v & 0xffffu), S.rs[r].n_groups, SELF_BLOCK, C.err)]);
              const int o = S.off[r];
              c = Bk.z & 0xffff;
              CK_RANGE(o + Bk.x, o + Bk.x + c, min(C.M, 1024), SELF_BLOCK, C.err);
              CK_RANGE(o + Bk.y, o + Bk.y + ((Bk.z >> 16) & 0xff), min(C.M, 1024), SELF_BLOCK, C.err);
              CK_RANGE(Bk.w, Bk.w + c, min(S.rs[r].md->n_masks, 65536), SELF_MASK, C.err);
              cl.sc[i] = (uint32_t)(o + Bk.x) | ((uint32_t)(o + Bk.y) << 10) | ((uint32_t)r << 20);
              cl.scn[i] = (uint16_t)Bk.w;
              cl.sck[i] = (uint8_t)(r * kMaxLinks + CK((Bk.z >> 24) & 15, S.rs[r].n_links, SELF_BLOCK, C.err));
            }
            base = scan_chunk(cl.pf, i, ns, c, base, lane);
          }
          if (lane == 0) cl.pf[ns] = base;
          __syncwarp();
          int it = 0;
          uint32_t nt = 0;
          for (int f = lane; f < base; f += kWarp) {
            while (cl.pf[it + 1] <= f) ++it;
            const uint32_t v = cl.sc[it];
            const int row = f - cl.pf[it];
            const float4 pa = P[(int)(v & 1023u) + row];
            // a row sphere clear of the column frame's bounding sphere is clear
            // of every column sphere
            nt += 1;
            if (!sph_hit(pa, S.BS[cl.sck[it]])) continue;
            const float4 *Pc = P + ((v >> 10) & 1023u);
            uint32_t mk = __ldg(&S.rs[v >> 20].masks[cl.scn[it] + row]);
            nt += (uint32_t)__popc(mk);
            while (mk) {
              const int c = __ffs(mk) - 1;
              mk &= mk - 1;
              hit |= sph_hit(pa, Pc[CK((int)((v >> 10) & 1023u) + c, C.M, SELF_MASK, C.err) - (int)((v >> 10) & 1023u)]);
            }
          }
          acc.tests += nt;
          __syncwarp();
        } else if (!hands_over<FULL, WS>() && cl.ns) {
          // self pairs from the pair list, one contiguous run per lane
          place_needed(C, S, xf, jj, lane, acc);
          const int ns = cl.ns;
          int base = 0;
          for (int i0 = 0; i0 < ns; i0 += kWarp) {
            const int i = i0 + lane;
            int c = 0;
            if (i < ns) c = cl.scn[i];
            base = scan_chunk(cl.pf, i, ns, c, base, lane);
          }
          if (lane == 0) cl.pf[ns] = base;
          __syncwarp();
          const int per = (base + kWarp - 1) / kWarp;
          int f = lane * per;
          const int fe = min(f + per, base);
          if (f < fe) {
            acc.tests += (uint32_t)(fe - f);
            for (int it = list_find(cl.pf, ns, f); f < fe; ++it) {
              const uint32_t v = cl.sc[it];
              const int r = (int)(v >> 16);
              const int ge = min(fe, cl.pf[it + 1]);
              const uint32_t *pr = S.rs[r].self + (int)(v & 0xffffu) - cl.pf[it];
              const float4 *Pr = P + S.off[r];
              CK_RANGE((int)(v & 0xffffu) + (f - cl.pf[it]), (int)(v & 0xffffu) + (ge - cl.pf[it]),
                 (S.rs[r].n_self + 3) & ~3, SELF_PAIR, C.err);
#pragma unroll 4
              for (; f < ge; ++f) {
                const uint32_t e = __ldg(&pr[f]);
                hit |= sph_hit(Pr[CK((int)(e & 0xffffu), S.rs[r].m, SELF_PAIR, C.err)],
                               Pr[CK((int)(e >> 16), S.rs[r].m, SELF_PAIR, C.err)]);
              }
            }
          }
          __syncwarp();
        }
      }
    }
    if (__any_sync(0xffffffffu, hit) && !exhaustive) return 1u;
  }
  if (!do_pairs) return __any_sync(0xffffffffu, hit) ? 1u : 0u;
  // robot-robot: every (robot pair, frame pair) as one flat range
  if (lane == 0) {
    cl.np = 0;
    cl.overflow = 0;
  }
  __syncwarp();
  // the phase's entries of the pair table (prioritized MV: the pairs (0, j),
  // listed first; pairs first: the adjacent pairs, listed first, or the rest);
  // frame pair g of table entry it: test the two frames' bounding spheres
  auto frame_pair = [&](int it, int g) {
    const uint32_t e = S.rp[CK(it, WS::kRobots * (WS::kRobots - 1) / 2, PAIRTAB, C.err)];
    const int i = CK((int)(e & 15u), n, PAIRTAB, C.err), j = CK((int)((e >> 4) & 15u), n, PAIRTAB, C.err);
    const int nj = (int)((e >> 8) & 15u);
    const int u = CK((g * (int)(e >> 16)) >> 12, S.rs[i].n_links, LINK, C.err);
    const int v = CK(g - u * nj, nj, LINK, C.err);
    const int k = i * kMaxLinks + u, k2 = j * kMaxLinks + v;
    const float4 bu = S.BS[k], bv = S.BS[k2];
    if (bu.w < 0.f || bv.w < 0.f) return;
    acc.tests += 1;
    if (sph_hit(bu, bv)) {
      push_cand(cl.pc, &cl.np, &cl.overflow, ((uint32_t)k << 8) | (uint32_t)k2);
      need_frame(cl, k);
      need_frame(cl, k2);
    }
  };
  if constexpr (WS::kLarge) {
    // large teams: frame pairs only for robot pairs whose enclosing spheres
    // overlap.  Robot r's sphere: center at the middle of its frame centers'
    // box, radius the largest distance to a frame sphere's far side, enlarged
    // by 1e-6 relative + 1e-4 m, so it holds every frame sphere with a margin
    // above the FP32 rounding of both tests: a frame pair whose spheres the
    // test finds overlapping always has its robot pair kept (same candidates).
    if (lane < n) {
      const float4 *bs = S.BS + lane * kMaxLinks;
      const int nl = S.rs[lane].n_links;
      float x0 = INFINITY, y0 = INFINITY, z0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, z1 = -INFINITY;
      for (int l = 0; l < nl; ++l) {
        const float4 b = bs[l];
        if (b.w < 0.f) continue;
        x0 = fminf(x0, b.x); y0 = fminf(y0, b.y); z0 = fminf(z0, b.z);
        x1 = fmaxf(x1, b.x); y1 = fmaxf(y1, b.y); z1 = fmaxf(z1, b.z);
      }
      float4 rs = make_float4(0.f, 0.f, 0.f, -1.f);
      if (x0 <= x1) {
        rs.x = 0.5f * (x0 + x1); rs.y = 0.5f * (y0 + y1); rs.z = 0.5f * (z0 + z1);
        float R = 0.f;
        for (int l = 0; l < nl; ++l) {
          const float4 b = bs[l];
          if (b.w < 0.f) continue;
          const float dx = b.x - rs.x, dy = b.y - rs.y, dz = b.z - rs.z;
          R = fmaxf(R, sqrtf(dx * dx + dy * dy + dz * dz) + b.w);
        }
        rs.w = R * (1.f + 1e-6f) + 1e-4f;
      }
      cl.rsph[CK(lane, WS::Cl::kCullR, ROBOT_CULL, C.err)] = rs;
    }
    __syncwarp();
    int nk = 0;
    for (int p0 = C.pr0; p0 < C.pr1; p0 += kWarp) {
      const int p = p0 + lane;
      bool keep = false;
      if (p < C.pr1) {
        const uint32_t e = S.rp[p];
        const float4 a = cl.rsph[e & 15u], b = cl.rsph[(e >> 4) & 15u];
        keep = a.w >= 0.f && b.w >= 0.f && sph_hit(a, b);
        acc.tests += 1;
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) cl.kept[CK(nk + __popc(m & ((1u << lane) - 1u)), WS::Cl::kCullP, ROBOT_CULL, C.err)] = (int16_t)p;
      nk += __popc(m);
    }
    __syncwarp();
    int base = 0;
    for (int i0 = 0; i0 < nk; i0 += kWarp) {
      const int i = i0 + lane;
      const int c = i < nk ? S.rpf[cl.kept[i] + 1] - S.rpf[cl.kept[i]] : 0;
      base = scan_chunk(cl.keptf, i, nk, c, base, lane);
    }
    if (lane == 0) cl.keptf[nk] = base;
    __syncwarp();
    int it = 0;
    for (int f = lane; f < base; f += kWarp) {
      while (cl.keptf[it + 1] <= f) ++it;
      frame_pair(cl.kept[it], f - cl.keptf[it]);
    }
  } else if (WS::kFPCap > 0 && C.fpt) {
    if (C.fpt == 1) {
      // the frame-pair table, built once per work item: entry e of robot-pair
      // entry p is its (e - fpf[p])-th pair (u, v) of frames holding spheres
      const int npr = C.prio ? n - 1 : n * (n - 1) / 2;
      const int ftot = S.fpf[npr];
      int p = 0;
      for (int e = lane; e < ftot; e += kWarp) {
        while (S.fpf[p + 1] <= e) ++p;
        const uint32_t r = S.rp[p];
        const int i = (int)(r & 15u), j = (int)((r >> 4) & 15u);
        const uint32_t mi = S.rs[i].md->frame_mask, mj = S.rs[j].md->frame_mask;
        const int nj = __popc(mj), g = e - S.fpf[p];
        const int ui = g / nj, vi = g - ui * nj;
        const int u = __fns(mi, 0, ui + 1), v = __fns(mj, 0, vi + 1);
        S.fp[CK(e, WS::kFPCap > 0 ? WS::kFPCap : 1, PAIRTAB, C.err)] =
            (uint16_t)((i * kMaxLinks + u) | ((j * kMaxLinks + v) << 8));
      }
      __syncwarp();
      if (lane == 0) C.fpt = 2;
      __syncwarp();
    }
    // the phase's frame pairs whose frames hold spheres, from the table
    const int ftot = S.fpf[C.pr1];
    for (int f = S.fpf[C.pr0] + lane; f < ftot; f += kWarp) {
      const uint32_t e = S.fp[f];
      const int k = (int)(e & 0xffu), k2 = (int)(e >> 8);
      acc.tests += 1;
      if (sph_hit(S.BS[k], S.BS[k2])) {
        push_cand(cl.pc, &cl.np, &cl.overflow, ((uint32_t)k << 8) | (uint32_t)k2);
        need_frame(cl, k);
        need_frame(cl, k2);
      }
    }
  } else if (hands_over<FULL, WS>()) {
    return kRedoState;   // more frame pairs than the table holds
  } else {
    const int ftot = S.rpf[C.pr1];
    int it = C.pr0;
    for (int f = S.rpf[C.pr0] + lane; f < ftot; f += kWarp) {
      while (S.rpf[it + 1] <= f) ++it;
      frame_pair(it, f - S.rpf[it]);
    }
  }
  __syncwarp();
  unsigned pm = 0;
  const int np = cl.np;
  if (hands_over<FULL, WS>() && cl.overflow) return kRedoState;
  if (!hands_over<FULL, WS>() && cl.overflow) {
    // every pair of the query's checked robots (a superset of the phase's
    // entries in the pairs-first order: an MV collision found there is one)
    need_all(cl, lane);
    place_needed(C, S, xf, jj, lane, acc);
    unsigned long long t = 0;
    pm = pairs_broad(C, S, P, lane, ffc, t);
    acc.tests += (uint32_t)t;
  } else if (np > 0) {
    place_needed(C, S, xf, jj, lane, acc);
    // flat (candidate, sphere of frame k) range; each entry tests frame k2
    int base = 0;
    for (int i0 = 0; i0 < np; i0 += kWarp) {
      const int i = i0 + lane;
      const int c = i < np ? frame_count(S, (int)(cl.pc[i] >> 8)) : 0;
      base = scan_chunk(cl.pf, i, np, c, base, lane);
    }
    if (lane == 0) cl.pf[np] = base;
    __syncwarp();
    const int per = (base + kWarp - 1) / kWarp;
    int f = lane * per;
    const int fe = min(f + per, base);
    if (f < fe) {
      for (int it = list_find(cl.pf, np, f); f < fe; ++it) {
        const uint32_t v = cl.pc[CK(it, kCand, CAND, C.err)];
        const int k = CK((int)(v >> 8), WS::kRobots * kMaxLinks, CAND, C.err);
        const int k2 = CK((int)(v & 0xffu), WS::kRobots * kMaxLinks, CAND, C.err);
        const int ge = min(fe, cl.pf[it + 1]);
        CK_RANGE(frame_first(S, k) + (f - cl.pf[it]), frame_first(S, k) + (ge - cl.pf[it]), C.M, SPHERE, C.err);
        const float4 *Pk = P + frame_first(S, k) - cl.pf[it];
        const int b0 = frame_first(S, k2), b1 = CK(b0 + frame_count(S, k2), C.M + 1, SPHERE, C.err);
        acc.tests += (uint32_t)((ge - f) * (b1 - b0));
        bool h = false;
        for (; f < ge; ++f) {
          const float4 pa = Pk[f];
#pragma unroll 4
          for (int b = b0; b < b1; ++b) h |= sph_hit(pa, P[b]);
        }
        if (h) pm = ffc ? max(pm, pair_code(pair_index(k / kMaxLinks, k2 / kMaxLinks, n))) : 1u;
      }
    }
  }
  if (ffc) return __reduce_max_sync(0xffffffffu, pm);
  return __any_sync(0xffffffffu, hit || pm != 0) ? 1u : 0u;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// adds a slice's per-lane broadphase statistics to the work item's
__device__ __forceinline__ void flush_acc(TileCtx &C, BroadAcc &acc, int lane) {
  const unsigned long long t = warp_sum((unsigned long long)acc.tests);
  const unsigned long long b = warp_sum((unsigned long long)acc.boxes);
  const unsigned long long cy = warp_sum((unsigned long long)acc.cyls);
  const unsigned long long p = warp_sum((unsigned long long)acc.placed);
  if (lane == 0) {
    C.tests += t;
    C.btests += b;
    C.ctests += cy;
    C.placed += p;
  }
  __syncwarp();
  acc.tests = acc.boxes = acc.placed = acc.cyls = 0u;
}

// clearance mode (exhaustive MV with min_clearance_out): direct formulas
template <class WS>
__device__ void clr_state(const TileCtx &C, const WS &S, const float4 *P, int lane, bool do_env, bool do_pairs,
                          float &minclr) {
  const int M = C.M;
  if (do_env && C.check_env) {
    for (int a = lane; a < C.env_rows; a += kWarp) {
      const float4 pa = P[a];
      const float4 w = make_float4(pa.x + S.ox, pa.y + S.oy, pa.z + S.oz, pa.w);
      for (int o = 0; o < C.env_ns; ++o) minclr = fminf(minclr, sph_clr(w, C.env_s[o]));
      for (int o = 0; o < C.env_nb; ++o)
        minclr = fminf(minclr, sqrtf(box_d2(w.x, w.y, w.z, C.box_lo[o], C.box_hi[o])) - w.w);
      for (int o = 0; o < C.env_nc; ++o)
        minclr = fminf(minclr, sqrtf(cyl_d2(w.x, w.y, w.z, __ldg(&C.cyl_a[o]), __ldg(&C.cyl_u[o]))) - w.w);
    }
    for (int r = 0; r < C.self_robots; ++r)
      for (int p = lane; p < S.rs[r].n_self; p += kWarp) {
        const uint32_t e = S.rs[r].self[p];
        minclr = fminf(minclr, sph_clr(P[S.off[r] + (e & 0xffffu)], P[S.off[r] + (e >> 16)]));
      }
  }
  if (do_pairs)
    for (int a = lane; a < S.off[C.pair_robots]; a += kWarp) {
      int r = 0;
      while (a >= S.off[r + 1]) ++r;
      const float4 pa = P[a];
      for (int b = S.off[r + 1]; b < M; ++b) minclr = fminf(minclr, sph_clr(pa, P[b]));
    }
}

template <bool FULL, class WS>
__device__ int slice_b(const BatchDev &B, TileCtx &C, WS &S, int k, int lane, float &minclr, bool do_env,
                       bool do_pairs) {
  const int n = C.n, M = C.M;
  const int CS = (kFkChains / n) < 1 ? 1 : (kFkChains / n);   // states per FK round (n chains each)
  float *xf = S.u.b.xf;
  float4 *P = S.u.b.P;
  float *K = S.u.b.K;
  const bool need_env = do_env && C.check_env;
  int found = C.ffc ? 0x7fffffff : 0;
  BroadAcc acc = {0u, 0u, 0u, 0u};
  const int nv = slice_valid(C, k);   // positions 0..nv-1 of the visiting order
  for (int j0 = 0; j0 < nv; j0 += CS) {
    // (state, robot) chains, three lanes per chain (one row of its frames
    // each), ten chains at a time
    for (int c = lane / 3; lane < 30 && c < CS * n; c += 10) {
      const int row = lane - 3 * (lane / 3);
      const int jj = j0 + c / n, r = c % n;
      if (jj < nv) {
        const int t = slice_state(C, k, slot_j(C, jj, nv));
        if (t <= C.T) {
          const RobotSlot &rs = S.rs[r];
          float q[MRV_MAX_DOF];
          const int T1 = S.itau[r];
          if (T1 >= 0) {
            // one segment from time 0 to T1 (the same arithmetic as interp)
            const float f = t >= T1 ? 0.f : (float)t / (float)T1;
            const float4 *A4 = reinterpret_cast<const float4 *>(S.ia[r]);
            const float4 *G4 = reinterpret_cast<const float4 *>(S.ig[r]);
            float av[MRV_MAX_DOF], gv[MRV_MAX_DOF];
#pragma unroll
            for (int h = 0; h < MRV_MAX_DOF / 4; ++h) {
              const float4 a4 = A4[h], g4 = G4[h];
              av[4 * h] = a4.x; av[4 * h + 1] = a4.y; av[4 * h + 2] = a4.z; av[4 * h + 3] = a4.w;
              gv[4 * h] = g4.x; gv[4 * h + 1] = g4.y; gv[4 * h + 2] = g4.z; gv[4 * h + 3] = g4.w;
            }
#pragma unroll
            for (int j = 0; j < MRV_MAX_DOF; ++j)
              if (j < rs.dof) q[j] = t >= T1 ? gv[j] : fmaf(gv[j] - av[j], f, av[j]);
          } else {
            int lo;
            interp_from(B, rs.w0, rs.w1, rs.dof, t, S.seg[r], q, &lo);
            if (row == 0) atomicMax(&S.seg[r], lo);
          }
          chain_row(B.models[rs.mdl], q, xf + CK(c, WS::kChains, CHAIN, C.err) * (kMaxLinks * 12), row);
        }
      }
    }
    if (lane == 0) C.chains += (unsigned long long)(min(CS, nv - j0) * n);   // FK chains (statistics)
    __syncwarp();
    for (int j = j0; j < j0 + CS && j < nv; ++j) {
      const int t = slice_state(C, k, slot_j(C, j, nv));
      if (lane == 0 && C.first_phase) C.states += 1;   // two-phase orders: counted in the first phase
      if (!FULL || (C.broad && !C.clr)) {
        // frame-level broadphase; spheres are placed only for the frames whose
        // bounding spheres overlap something, then resolved exactly (the
        // default instance has this path only)
        link_spheres(C, S, xf, j - j0, lane);
        __syncwarp();
        const unsigned res = broad_state<FULL>(C, S, xf, j - j0, lane, need_env, do_pairs, acc);
        __syncwarp();
        if (hands_over<FULL, WS>() && res == kRedoState) {
          flush_acc(C, acc, lane);
          return kSliceRedo;
        }
        if (res) {
          if (!C.ffc) {
            if (!C.exhaustive) {
              flush_acc(C, acc, lane);
              return 1;
            }
            found = 1;
          } else {
            const int key = code_key(t, res);
            if (!C.exhaustive) {
              flush_acc(C, acc, lane);
              return key;
            }
            if (key < found) found = key;
          }
        }
        continue;
      }
      if (lane == 0) C.placed += (unsigned long long)M;
      // sphere placement relative to the query origin, robot by robot
      float c2 = 0.f, cw2 = 0.f;
      for (int r = 0; r < n; ++r) {
        const float *Xr = xf + CK((j - j0) * n + r, WS::kChains, CHAIN, C.err) * (kMaxLinks * 12);
        const float4 *sph = S.rs[r].spheres;
        const int32_t *lnk = S.rs[r].links;
        const int m = S.rs[r].m, a0 = CK(S.off[r] + S.rs[r].m, C.M + 1, SPHERE, C.err) - S.rs[r].m;
#pragma unroll 4
        for (int kk = lane; kk < m; kk += kWarp) {
          const float4 s = __ldg(&sph[kk]);
          const float3 w = frame_apply(Xr + CK(__ldg(&lnk[kk]), S.rs[r].n_links, LINK, C.err) * 12, s.x, s.y, s.z);
          const float wx = w.x, wy = w.y, wz = w.z;
          const float px = wx - S.ox, py = wy - S.oy, pz = wz - S.oz;
          P[a0 + kk] = make_float4(px, py, pz, s.w);
          const float pp = fmaf(px, px, fmaf(py, py, pz * pz));
          K[a0 + kk] = fmaf(-s.w, s.w, pp);
          c2 = fmaxf(c2, pp);
          cw2 = fmaxf(cw2, fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
        }
      }
      c2 = warp_max(c2);
      if (need_env) cw2 = warp_max(cw2);
      __syncwarp();
      const float eps = kEpsU * (c2 + C.rho2);
      if (!C.ffc) {
        bool hit = false;
        if (C.clr) {
          clr_state(C, S, P, lane, do_env, do_pairs, minclr);
          hit = minclr < 0.f;
        } else if (need_env) {
          // combined order (Alg. 1): env + self of every robot, then pairs
          hit = env_mv(C, S, P, K, lane, cw2, eps);
          if (!C.exhaustive && __any_sync(0xffffffffu, hit)) {
            if (lane == 0) {
              C.tests += (unsigned long long)(C.envtests + C.boxtests + C.cyltests);
              C.btests += (unsigned long long)C.boxtests;
              C.ctests += (unsigned long long)C.cyltests;
            }
            return 1;
          }
        }
        if (need_env && lane == 0) {
          C.tests += (unsigned long long)(C.envtests + C.boxtests + C.cyltests);
          C.btests += (unsigned long long)C.boxtests;
          C.ctests += (unsigned long long)C.cyltests;
        }
        if (do_pairs) {
          if (!C.clr) {
            if (C.pr0 == 0 && C.rangetests == C.pairtests) hit |= pairs_mv(P, K, S.off, n, M, lane, eps, C.pair_robots);
            else hit |= pairs_list_mv(P, K, S, C.pr0, C.pr1, lane, eps);
          }
          if (lane == 0) C.tests += (unsigned long long)C.rangetests;
        }
        if (__any_sync(0xffffffffu, hit)) {
          if (!C.exhaustive) return 1;
          found = 1;
        }
      } else {
        unsigned pm = pairs_ffc(P, K, S.off, n, lane, eps);
        if (lane == 0) C.tests += (unsigned long long)C.pairtests;
        pm = __reduce_max_sync(0xffffffffu, pm);
        if (pm) {
          const int key = code_key(t, pm);
          if (!C.exhaustive) return key;
          if (key < found) found = key;   // states run in increasing t
        }
      }
      __syncwarp();
    }
    __syncwarp();
  }
  if (!FULL || (C.broad && !C.clr)) flush_acc(C, acc, lane);
  return found;
}

// ---------------------------------------------------------------------------
// the persistent work-stealing kernel
// ---------------------------------------------------------------------------

// s states of query q (s in two's complement: negative to take them back)
// and the method's dense work of those states, added to the statistics:
// every test and placement of the query's flavor, whatever the broadphase
// skipped
__device__ __forceinline__ void add_state_stats(const BatchDev &B, int q, unsigned long long s) {
  const QueryDev *Qd = B.q + q;   // read here: not held in registers over the item
  const unsigned long long bt = (unsigned long long)__ldg(&Qd->boxtests);
  const unsigned long long ct = (unsigned long long)__ldg(&Qd->cyltests);
  const int nch = __ldg(&Qd->nchain);
  atomicAdd(&B.stats[9], s * (unsigned long long)(__ldg(&Qd->pairtests) + __ldg(&Qd->envtests)));
  if (bt) atomicAdd(&B.stats[10], s * bt);
  if (ct) atomicAdd(&B.stats[11], s * ct);
  if (nch) {
    atomicAdd(&B.stats[12], s * (unsigned long long)__ldg(&Qd->njoint));
    atomicAdd(&B.stats[13], s * (unsigned long long)nch);
  }
  atomicAdd(&B.stats[14], s * (unsigned long long)__ldg(&Qd->M));
  atomicAdd(&B.stats[0], s);
}

template <bool FULL, class WS>
__device__ void run_chunk(const BatchDev &B, WS &S, int q, int c, int lane) {
  const QueryDev Q = B.q[q];
  if (!(B.flags & MRV_EXHAUSTIVE)) {
    // a verdict reached since the item was claimed: skip the staging too
    int stop = 0;
    if (lane == 0)
      stop = !(Q.bits & 1u) ? *(volatile int *)&B.q_hit[q] != 0
                            : *(volatile int *)&B.q_best[q] < (min(c * Q.cte * Q.spt, Q.T) << kKeyShift);
    if (__shfl_sync(0xffffffffu, stop, 0)) return;
  }
  TileCtx &C = S.ctx;   // kept in shared memory: read where used, not held in registers
  __syncwarp();
  C.err = B.err;
  C.q = q; C.T = Q.T; C.n = CK(Q.n - 1, WS::kRobots, SLOTS, B.err) + 1;
  C.M = CK(Q.M - 1, WS::kSpheres, SPHERE, B.err) + 1; C.nb = Q.ntiles;
  C.ffc = Q.bits & 1u;
  C.check_env = (!C.ffc) && (B.flags & MRV_CHECK_ENV);
  C.exhaustive = (B.flags & MRV_EXHAUSTIVE) ? 1 : 0;
  C.split = Q.split; C.spt = Q.spt; C.nslices = Q.nslices;
  C.broad = (B.flags & MRV_NO_BROADPHASE) ? 0 : 1;
  C.lin = (C.ffc || (B.flags & MRV_LINEAR)) ? 1 : 0;
  C.prio = (!C.ffc && (B.flags & MRV_PRIORITY)) ? 1 : 0;
  C.clr = (FULL && B.clr && !C.ffc) ? 1 : 0;
  C.env_ns = 0; C.env_nb = 0; C.env_s = nullptr; C.env_k = nullptr; C.box_lo = nullptr; C.box_hi = nullptr;
  C.env = nullptr;
  C.env_nc = 0; C.cyl_a = nullptr; C.cyl_u = nullptr;
  C.env_c2 = 0.f; C.env_r2 = 0.f; C.rho2 = Q.rho2;
  if (C.check_env && Q.env >= 0) {
    const EnvDev &E = B.envs[Q.env];
    C.env = &E;
    C.env_nc = E.n_cyl; C.cyl_a = E.cyl_a; C.cyl_u = E.cyl_u;
    C.env_ns = E.n_spheres; C.env_nb = E.n_aabbs; C.env_s = E.spheres; C.env_k = E.sphere_k;
    C.box_lo = E.box_lo; C.box_hi = E.box_hi; C.env_c2 = E.c2max; C.env_r2 = E.r2max;
  }
  C.pairtests = Q.pairtests; C.envtests = Q.envtests; C.boxtests = Q.boxtests; C.cyltests = Q.cyltests;
  C.tests = 0; C.btests = 0; C.states = 0; C.chains = 0; C.placed = 0; C.ctests = 0;
  // stage the query's robots; origin of the relative frame = robot 0's base
  const int s0 = B.q_robot_off[q];
  uint32_t fm = 0;   // this lane's robot: frames holding spheres
  if (lane < C.n) {
    const int id = CK(B.slot_robot_id[CK(s0 + lane, B.n_slots, SLOTS, B.err)], B.n_models, SLOTS, B.err);
    const ModelDev &m = B.models[id];
    fm = m.frame_mask;
    RobotSlot rs;
    rs.spheres = m.spheres; rs.links = m.sphere_link; rs.self = m.self_pairs; rs.rects = m.self_rects; rs.md = &m;
    rs.masks = m.self_masks;
    rs.mdl = id; rs.m = m.n_spheres; rs.dof = m.dof; rs.kind = m.kind; rs.n_self = m.n_self;
    rs.w0 = B.slot_wp_off[s0 + lane]; rs.w1 = B.slot_wp_off[s0 + lane + 1]; rs.n_rects = m.n_rects;
    rs.n_links = m.n_links; rs.n_groups = m.n_groups;
    rs.nfr = (int16_t)__popc(fm);
#pragma unroll
    for (int l = 0; l < kMaxLinks + 2; ++l) rs.ls[l] = (int16_t)(l <= m.n_links ? m.link_start[l] : m.n_spheres);
    S.rs[lane] = rs;
    S.seg[lane] = rs.w0;
    if (rs.w1 - rs.w0 == 2) {
      const int w = CK(rs.w0 + 1, B.n_waypoints, WAYPOINT, B.err);
      const float *a = B.waypoints + (size_t)(w - 1) * B.wp_stride;
      S.itau[lane] = B.slot_tau[w];
#pragma unroll
      for (int j = 0; j < MRV_MAX_DOF; ++j)
        if (j < rs.dof) {
          S.ia[lane][j] = a[j];
          S.ig[lane][j] = a[B.wp_stride + j];
        }
    } else {
      S.itau[lane] = -1;
    }
    if (lane == 0) { S.ox = m.base[3]; S.oy = m.base[7]; S.oz = m.base[11]; }
  }
  {
    // the frame slots holding spheres, robot by robot (lane r writes robot
    // r's at the prefix of the counts); every other slot's bounding sphere
    // is "none" for the whole item
    const int cnt = __popc(fm);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int pos = incl - cnt;
    while (fm) {
      const int l = __ffs(fm) - 1;
      fm &= fm - 1;
      S.ef[CK(pos++, WS::kRobots * kMaxLinks, FRAME_SLOT, B.err)] = (uint8_t)(lane * kMaxLinks + l);
    }
    const int tot = __shfl_sync(0xffffffffu, incl, kWarp - 1), n0 = __shfl_sync(0xffffffffu, incl, 0);
    for (int k = lane; k < C.n * kMaxLinks; k += kWarp) S.BS[k] = make_float4(0.f, 0.f, 0.f, -1.f);
    if (lane == 0) {
      C.nef = tot;
      C.nef_env = C.prio ? n0 : tot;
    }
  }
  __syncwarp();
  if (lane == 0) {
    int acc = 0;
    S.off[0] = 0;
    for (int r = 0; r < C.n; ++r) { acc += S.rs[r].m; S.off[r + 1] = acc; }
    C.env_rows = C.prio ? S.off[1] : C.M;
    C.self_robots = C.prio ? 1 : C.n;
    C.pair_robots = C.prio ? 1 : C.n - 1;
    int blk = 1;
    for (int r = 0; r < C.n; ++r) blk &= (S.rs[r].n_groups == 0 || S.rs[r].masks != nullptr);
    C.self_blk = blk;
    // pairs in (i, j) order; pairs-first MV lists the adjacent pairs first
    int p = 0, f = 0, ff = 0;
    const bool pf = !C.ffc && Q.nadj > 0;
    const uint32_t *adj = B.q[q].adj;   // read in place (a copy indexed at run time would live in local memory)
    for (int pass = pf ? 0 : 1; pass < 2; ++pass)
      for (int i = 0, pi = 0; i < C.n; ++i)
        for (int j = i + 1; j < C.n; ++j, ++pi) {
          if (pf && (((__ldg(&adj[pi >> 5]) >> (pi & 31)) & 1u) != (pass == 0 ? 1u : 0u))) continue;
          const int nj = S.rs[j].n_links;
          const int pc = CK(p, WS::kRobots * (WS::kRobots - 1) / 2, PAIRTAB, B.err);
          S.rp[pc] = (uint32_t)(i | j << 4 | nj << 8) | ((uint32_t)((4096 + nj - 1) / nj) << 16);
          S.rpf[pc] = (int16_t)CK(f, 32768, PAIRTAB_PREFIX, B.err);
          S.fpf[pc] = (int16_t)ff;
          f += S.rs[i].n_links * S.rs[j].n_links;
          ff += S.rs[i].nfr * S.rs[j].nfr;
          ++p;
        }
    S.rpf[CK(p, WS::kRobots * (WS::kRobots - 1) / 2 + 1, PAIRTAB, B.err)] = (int16_t)CK(f, 32768, PAIRTAB_PREFIX, B.err);
    S.fpf[p] = (int16_t)min(ff, 32767);
    // the table pays for its construction once an item spans 8 states or more
    C.fpt = (WS::kFPCap > 0 && ff <= WS::kFPCap && (WS::kClass == 0 || Q.cte * Q.spt >= 8)) ? 1 : 0;
  }
  __syncwarp();
  const int total = Q.nslices * Q.nphase;
  const int k0 = c * Q.cte;
  const int k1 = min(k0 + Q.cte, total);
  float minclr = INFINITY;
  for (int kt = k0; kt < k1; ++kt) {
    const int phase = Q.nphase == 2 ? kt / Q.nslices : -1;
    const int k = Q.nphase == 2 ? kt - phase * Q.nslices : kt;
    // combined: obstacles + self and every pair; hierarchical: obstacles +
    // self, then the pairs; pairs first: the adjacent pairs, then obstacles +
    // self and the other pairs
    const bool pf = Q.nadj > 0;
    const bool do_env = pf ? phase == 1 : phase != 1;
    const int npr = C.prio ? C.n - 1 : C.n * (C.n - 1) / 2;
    const int pr0 = (pf && phase == 1) ? Q.nadj : 0;
    const int pr1 = pf ? (phase == 0 ? Q.nadj : npr) : (phase == 0 ? 0 : npr);
    const bool do_pairs = pr1 > pr0;
    if (lane == 0) {
      C.pr0 = pr0;
      C.pr1 = pr1;
      C.first_phase = phase <= 0;
      C.rangetests = !pf ? Q.pairtests : (phase == 0 ? Q.adjtests : Q.pairtests - Q.adjtests);
    }
    __syncwarp();
    if (!C.exhaustive) {
      // one lane reads the query's shared verdict so the warp decides together
      int stop = 0;
      if (lane == 0)
        stop = !C.ffc ? *(volatile int *)&B.q_hit[q] != 0
                      : *(volatile int *)&B.q_best[q] < (min(slice_state(C, k, 0), C.T) << kKeyShift);
      if (__shfl_sync(0xffffffffu, stop, 0)) break;
    }
    const int res = ((FULL || WS::kClass != 0) && (Q.bits & 2u)) ? slice_a<FULL>(B, C, S, k, lane, minclr, do_env, do_pairs)
                                            : slice_b<FULL>(B, C, S, k, lane, minclr, do_env, do_pairs);
    if (hands_over<FULL, WS>() && res == kSliceRedo) {
      // the query goes to the full instance's pass, listed once; that pass
      // reruns every item of it (the checks of a state are idempotent)
      if (lane == 0 && atomicExch(&B.redo_flag[q], 1) == 0)
        B.redo[CK(atomicAdd(&B.counters[kCtrRedo], 1), B.n_queries, QUERY, B.err)] = q;
      break;
    }
    if (!C.ffc) {
      if (res) {
        if (lane == 0) atomicExch(&B.q_hit[q], 1);
        if (!C.exhaustive) break;
      }
    } else if (res != 0x7fffffff) {
      if (lane == 0) atomicMin(&B.q_best[q], res);
      if (!C.exhaustive) break;
    }
    __syncwarp();
  }
  if (FULL && C.clr) {
    for (int o = 16; o > 0; o >>= 1) minclr = fminf(minclr, __shfl_xor_sync(0xffffffffu, minclr, o));
    if (lane == 0) atomicMin((int *)&B.q_minclr[q], f2ord(minclr));
  }
  __syncwarp();
  if (lane == 0) {
    // the states this item checked (each state counts once, in its first
    // phase) and the method's dense work of them; the default instances
    // also keep each query's count, which the full instance's pass takes
    // back before it reruns a query handed over
    if (C.states) {
      add_state_stats(B, q, C.states);
      if (hands_over<FULL, WS>()) atomicAdd(&B.q_states[q], (int)C.states);
    }
    atomicAdd(&B.stats[1], C.tests);
    atomicAdd(&B.stats[5], C.btests);
    atomicAdd(&B.stats[8], C.ctests);
    atomicAdd(&B.stats[6], C.chains);
    atomicAdd(&B.stats[7], C.placed);
  }
  __syncwarp();
}

// The persistent kernel.  Launch bounds: 512 threads per SM for the
// small-team layout (at most 128 registers, 16 warps sharing an SM) and 384
// for the others (168 registers; 12 warps of the team layout).  The instance
// of layout WS takes the work items of its class; FULL selects the instance
// with every path (see hands_over), and q_single one query per launch
// (>= 0) or the full instance's pass over the handed-over queries
// (kRedoPass).
template <bool FULL, class WS>
__global__ void __launch_bounds__(WS::kMaxThreads, 1) k_main(BatchDev B, int q_single) {
  extern __shared__ float4 smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  WS &S = *reinterpret_cast<WS *>(reinterpret_cast<char *>(smem_raw) + warp * warp_smem_bytes<WS>());
  constexpr int cls = WS::kClass;
  const long long t_start = clock64();
  if (q_single == kRedoPass) {
    // the full instance (large-team layout, which holds any query) reruns
    // every item of the queries the default instances handed over, one
    // query per warp at a time
    if constexpr (FULL) {
      const int n = *(volatile int *)&B.counters[kCtrRedo];
      for (;;) {
        int e = 0;
        if (lane == 0) e = atomicAdd(&B.counters[kCtrRedoClaim], 1);
        e = __shfl_sync(0xffffffffu, e, 0);
        if (e >= n) break;
        const int q = CK(B.redo[CK(e, B.n_queries, QUERY, B.err)], B.n_queries, QUERY, B.err);
        if (lane == 0) {
          // the states the default instance counted for q are checked again here
          const int sp = atomicExch(&B.q_states[q], 0);
          if (sp) add_state_stats(B, q, (unsigned long long)(-(long long)sp));
        }
        __syncwarp();
        const int nch = B.q[q].nchunks;
        for (int c = 0; c < nch; ++c) run_chunk<FULL>(B, S, q, c, lane);
        if (lane == 0) atomicAdd(&B.stats[15], 1ull);
      }
    }
    return;
  }
  if (q_single >= 0) {
    // one launch per query: warp w of block x takes items x*warps + w, ...
    const QueryDev Q = B.q[q_single];
    if (Q.bits & 4u) return;
    for (int c = blockIdx.x * (blockDim.x >> 5) + warp; c < Q.nchunks; c += gridDim.x * (blockDim.x >> 5))
      run_chunk<FULL>(B, S, q_single, c, lane);
    return;
  }
  const int n_items = B.counters[kCtrItems(cls)];
  if (n_items == 0) return;
  const int *level_start = B.level_start + cls * (kMaxLevels + 1);
  const int qbase = B.counters[kCtrFirst(cls)];   // first sorted position of the class
  const bool skip_dead = !(B.flags & MRV_EXHAUSTIVE);
  unsigned long long items = 0;
  // Items are claimed g at a time.  Lane l < g resolves item base + l (level,
  // query) and whether its query already has a verdict that makes it dead
  // (MV: any collision; FFC: a conflict before the item's first state).  g
  // doubles while whole claims are settled and drops back to 1 at live work,
  // so live items are still spread one per claim.
  int g = 1;
  for (;;) {
    // the abort flag is read together with the claim (both round trips at once)
    int base = 0, aborted = 0;
    if (lane == 0) {
      base = atomicAdd(&B.counters[kCtrClaim(cls)], g);
      aborted = *(volatile int *)&B.counters[kCtrAbort];
#ifdef MRV_CHECKED
      aborted |= (*(volatile uint32_t *)B.err & kErrChecked) != 0u;   // stop at a failed index check
#endif
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_items) break;
    // a warp whose clock budget runs out raises the abort flag, so every
    // other warp stops at its next claim instead of at its own budget
    int halt = 0;
    if (lane == 0) {
      if (aborted) halt = 1;
      else if (B.clock_budget > 0 && clock64() - t_start > B.clock_budget) halt = 2;
      if (halt) atomicOr(B.err, halt == 1 ? kErrAbort : kErrTimeout);
      if (halt == 2) atomicExch(&B.counters[kCtrAbort], 1);
    }
    if (__shfl_sync(0xffffffffu, halt, 0)) break;
    const int idx = base + lane;
    int q = 0, lvl = 0;
    bool live = false;
    if (lane < g && idx < n_items) {
      int lo = 0, hi = kMaxLevels - 1;   // level: last c with level_start[c] <= idx
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&level_start[mid]) <= idx) lo = mid;
        else hi = mid - 1;
      }
      lvl = lo;
      q = __ldg(&B.sorted[CK(qbase + idx - __ldg(&level_start[lo]), B.n_queries, SORTED, B.err)]);
      q = CK(q, B.n_queries, QUERY, B.err);
      if (!skip_dead) {
        live = true;
      } else {
        // MV: any collision ends the query.  FFC: only a conflict before
        // the item's first state makes it dead (another warp may record a
        // later item's conflict between this claim and this check)
        const int best = *(volatile int *)&B.q_best[q];
        live = *(volatile int *)&B.q_hit[q] == 0 &&
               (best == 0x7fffffff ||
                best >= (min(lo * __ldg(&B.q[q].cte) * __ldg(&B.q[q].spt), __ldg(&B.q[q].T)) << kKeyShift));
      }
    }
    unsigned live_mask = __ballot_sync(0xffffffffu, live);
    g = live_mask ? 1 : min(2 * g, kWarp);
    while (live_mask) {
      const int src = __ffs(live_mask) - 1;
      live_mask &= live_mask - 1;
      const int qq = __shfl_sync(0xffffffffu, q, src), ll = __shfl_sync(0xffffffffu, lvl, src);
      run_chunk<FULL>(B, S, qq, ll, lane);
      ++items;
    }
  }
  if (lane == 0 && items) atomicAdd(&B.stats[4], items);
}

// results: MV -> valid byte (+ min clearance), FFC -> (t, i, j)
__global__ void k_finish(BatchDev B, uint8_t *valid_out, float *minclr_out, mrv_conflict *conf_out, int *counts) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B.n_queries) return;
  const QueryDev Q = B.q[q];
  if (!(Q.bits & 1u)) {
    const int v = (!(Q.bits & 4u) && B.q_hit[q] == 0) ? 1 : 0;
    if (valid_out) valid_out[q] = (uint8_t)v;
    if (minclr_out) minclr_out[q] = ord2f(__float_as_int(B.q_minclr[q]));
    if (v) atomicAdd(&counts[0], 1);
  } else {
    mrv_conflict c = {-1, -1, -1};
    const int key = B.q_best[q];
    if (key != 0x7fffffff && !(Q.bits & 4u)) {
      c.t = key >> kKeyShift;
      int p = key & ((1 << kKeyShift) - 1), i = 0;
      while (i < Q.n - 1 && p >= Q.n - 1 - i) { p -= Q.n - 1 - i; ++i; }
      c.i = CK(i, Q.n, FINISH_PAIR, B.err);
      c.j = CK(i + 1 + p, Q.n, FINISH_PAIR, B.err);
      atomicAdd(&counts[1], 1);
    }
    if (conf_out) conf_out[q] = c;
  }
}

// ---------------------------------------------------------------------------
// per-sphere clearance diagnostic: block = one listed timestep
// ---------------------------------------------------------------------------
__global__ void k_clearance(BatchDev B, int q, const int32_t *ts, int nt, int check_env, float *out) {
  __shared__ float4 P[MRV_MAX_QUERY_SPHERES];
  __shared__ float xf[MRV_MAX_ROBOTS * kMaxLinks * 12];
  __shared__ RobotSlot rs[MRV_MAX_ROBOTS];
  __shared__ int off[MRV_MAX_ROBOTS + 1];
  const int k = blockIdx.x;
  if (k >= nt) return;
  const QueryDev Q = B.q[q];
  if (Q.bits & 4u) return;
  const int t = ts[k];
  if (t < 0 || t > Q.T) {
    if (threadIdx.x == 0) atomicOr(B.err, kErrSteps);
    return;
  }
  const int s0 = B.q_robot_off[q];
  if (threadIdx.x < Q.n) {
    const int id = B.slot_robot_id[s0 + threadIdx.x];
    const ModelDev &m = B.models[id];
    RobotSlot r;
    r.spheres = m.spheres; r.links = m.sphere_link; r.self = m.self_pairs; r.rects = m.self_rects; r.md = &m;
    r.mdl = id; r.m = m.n_spheres; r.dof = m.dof; r.kind = m.kind; r.n_self = m.n_self;
    r.w0 = B.slot_wp_off[s0 + threadIdx.x]; r.w1 = B.slot_wp_off[s0 + threadIdx.x + 1]; r.n_rects = m.n_rects;
    rs[threadIdx.x] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    off[0] = 0;
    for (int r = 0; r < Q.n; ++r) { acc += rs[r].m; off[r + 1] = acc; }
  }
  if (threadIdx.x < Q.n) {
    float qq[MRV_MAX_DOF];
    const RobotSlot &r = rs[threadIdx.x];
    interp(B, r.w0, r.w1, r.dof, t, qq);
    chain_frames(B.models[r.mdl], qq, xf + threadIdx.x * kMaxLinks * 12);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < Q.M; a += blockDim.x) {
    int r = 0;
    while (a >= off[r + 1]) ++r;
    const int i = a - off[r];
    const float4 s = rs[r].spheres[i];
    const float *X = xf + r * kMaxLinks * 12 + CK(rs[r].links[i], kMaxLinks, LINK, B.err) * 12;
    P[CK(a, MRV_MAX_QUERY_SPHERES, CLEAR_OUT, B.err)] = make_float4(fmaf(X[0], s.x, fmaf(X[1], s.y, fmaf(X[2], s.z, X[3]))),
                       fmaf(X[4], s.x, fmaf(X[5], s.y, fmaf(X[6], s.z, X[7]))),
                       fmaf(X[8], s.x, fmaf(X[9], s.y, fmaf(X[10], s.z, X[11]))), s.w);
  }
  __syncthreads();
  const EnvDev *E = (check_env && Q.env >= 0) ? &B.envs[Q.env] : nullptr;
  for (int a = threadIdx.x; a < Q.M; a += blockDim.x) {
    int r = 0;
    while (a >= off[r + 1]) ++r;
    const float4 pa = P[a];
    float m = INFINITY;
    for (int bb = 0; bb < Q.M; ++bb)
      if (bb < off[r] || bb >= off[r + 1]) m = fminf(m, sph_clr(pa, P[bb]));
    if (check_env) {
      if (E) {
        for (int o = 0; o < E->n_spheres; ++o) m = fminf(m, sph_clr(pa, E->spheres[o]));
        for (int o = 0; o < E->n_aabbs; ++o)
          m = fminf(m, sqrtf(box_d2(pa.x, pa.y, pa.z, E->box_lo[o], E->box_hi[o])) - pa.w);
        for (int o = 0; o < E->n_cyl; ++o) m = fminf(m, sqrtf(cyl_d2(pa.x, pa.y, pa.z, E->cyl_a[o], E->cyl_u[o])) - pa.w);
      }
      const int li = a - off[r];
      for (int p = 0; p < rs[r].n_self; ++p) {
        const int ex = CK((int)(rs[r].self[p] & 0xffffu), rs[r].m, CLEAR_OUT, B.err);
        const int ey = CK((int)(rs[r].self[p] >> 16), rs[r].m, CLEAR_OUT, B.err);
        if (ex == li) m = fminf(m, sph_clr(pa, P[off[r] + ey]));
        else if (ey == li) m = fminf(m, sph_clr(pa, P[off[r] + ex]));
      }
    }
    // spheres are stored sorted by frame; the output keeps the caller's order
    out[(size_t)k * Q.M + off[r] + CK(rs[r].md->perm[a - off[r]], rs[r].m, CLEAR_OUT, B.err)] = m;
  }
}

// ---------------------------------------------------------------------------
// host-side launch wrappers
// ---------------------------------------------------------------------------

size_t main_smem_bytes(int warps, int cls) {
  const size_t per = cls == 2 ? warp_smem_bytes<WarpSmemLarge>()
                              : (cls == 1 ? warp_smem_bytes<WarpSmemTeam>() : warp_smem_bytes<WarpSmemSmall>());
  return per * (size_t)warps;
}

int large_warps() { return kLargeWarps; }

cudaError_t launch_prepare(const BatchDev &B, cudaStream_t st) {
  if (B.n_queries > 0) {
    const int th = 128, bl = (B.n_queries + th - 1) / th;
    k_prep<<<bl, th, 0, st>>>(B);
  }
  k_levels<<<1, kLevelThreads, 0, st>>>(B);
  if (B.n_queries > 0) {
    const int th = 256, bl = (B.n_queries + th - 1) / th;
    k_scatter<<<bl, th, 0, st>>>(B);
  }
  return cudaGetLastError();
}

// The dynamic shared memory limit of k_main is a process-wide attribute (per
// device): it is raised once to what the largest block (12 warps of the
// small-team and team layouts, kLargeWarps of the large-team layout) needs,
// so launches with fewer warps on other threads never see it shrink under
// them.
template <class WS>
static cudaError_t set_attrs_of(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_main<false, WS>, a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_main<true, WS>, a, bytes);
  return e;
}

cudaError_t set_main_attrs(int warps) {
  (void)warps;
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static bool done[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  e = set_attrs_of<WarpSmemSmall>((int)main_smem_bytes(12, 0));
  if (e == cudaSuccess) e = set_attrs_of<WarpSmemTeam>((int)main_smem_bytes(12, 1));
  if (e == cudaSuccess) e = set_attrs_of<WarpSmemLarge>((int)main_smem_bytes(kLargeWarps, 2));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

template <class WS>
static cudaError_t occupancy_of(int warps, bool full, int *out) {
  const size_t smem = main_smem_bytes(warps, WS::kClass);
  return full ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_main<true, WS>, warps * 32, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_main<false, WS>, warps * 32, smem);
}

cudaError_t max_blocks_per_sm(int warps, bool full, int cls, int *out) {
  set_main_attrs(warps);
  if (cls == 2) return occupancy_of<WarpSmemLarge>(warps, full, out);
  if (cls == 1) return occupancy_of<WarpSmemTeam>(warps, full, out);
  return occupancy_of<WarpSmemSmall>(warps, full, out);
}

// full: the instance with every path (the runs that ask for minimum
// clearances or name MRV_NO_BROADPHASE); otherwise the broadphase-only one
template <class WS>
static void launch_of(const BatchDev &B, int grid, int warps, bool full, int q_single, cudaStream_t st) {
  const size_t smem = main_smem_bytes(warps, WS::kClass);
  if (full) k_main<true, WS><<<grid, warps * 32, smem, st>>>(B, q_single);
  else k_main<false, WS><<<grid, warps * 32, smem, st>>>(B, q_single);
}

cudaError_t launch_main(const BatchDev &B, int grid, int warps, bool full, int cls, int q_single, cudaStream_t st) {
  if (cls == 2) launch_of<WarpSmemLarge>(B, grid, warps, full, q_single, st);
  else if (cls == 1) launch_of<WarpSmemTeam>(B, grid, warps, full, q_single, st);
  else launch_of<WarpSmemSmall>(B, grid, warps, full, q_single, st);
  return cudaGetLastError();
}

cudaError_t launch_finish(const BatchDev &B, uint8_t *valid, float *minclr, mrv_conflict *conf, int *counts,
                          cudaStream_t st) {
  if (B.n_queries == 0) return cudaSuccess;
  const int th = 256, bl = (B.n_queries + th - 1) / th;
  k_finish<<<bl, th, 0, st>>>(B, valid, minclr, conf, counts);
  return cudaGetLastError();
}

cudaError_t launch_clearance(const BatchDev &B, int q, const int32_t *ts, int nt, int check_env, float *out,
                             cudaStream_t st) {
  if (nt <= 0) return cudaSuccess;
  k_clearance<<<nt, 128, 0, st>>>(B, q, ts, nt, check_env, out);
  return cudaGetLastError();
}

}  // namespace mrv
