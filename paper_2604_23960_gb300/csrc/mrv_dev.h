// Device-side data layout shared by the host runtime and the kernels.
//
// Everything the kernels read lives in device memory owned by the context:
//   ModelDev  one entry per uploaded robot model (indexed by robot id); DH
//             rows are pre-split into cos/sin of alpha so the per-state chain
//             needs one sincosf per joint.
//   EnvDev    one entry per uploaded obstacle set (indexed by env slot).
//   BatchDev  the ragged CSR batch (caller arrays or staged copies) plus the
//             per-query / per-slot arrays derived on the device.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include "../../include/mrv.h"

// functions used by both the host runtime (g++) and the kernels (nvcc)
#ifdef __CUDACC__
#define MRV_HD __host__ __device__
#else
#define MRV_HD
#endif

namespace mrv {

constexpr int kWarp = 32;             // lanes per tile (the GPU's batch width W)
constexpr int kMaxLinks = MRV_MAX_DOF + 2;  // frames 0..dof+1
constexpr int kMaxLevels = 256;       // work levels (work items per query)
constexpr int kEnvIdBase = 1 << 20;   // env ids = kEnvIdBase + env slot
constexpr int kFkChains = 8;          // (state, robot) chains per FK round
// Work classes, one persistent-kernel instance (per-warp shared-memory
// layout) each: class 0 (small teams) up to kTeamRobots robots and
// kSmallSpheres spheres, 16 warps per SM; class 1 (teams) up to kTeamRobots
// robots and kTeamSpheres spheres, 12 warps per SM; class 2 (large teams) up
// to MRV_MAX_ROBOTS robots and MRV_MAX_QUERY_SPHERES spheres.  Each class has
// its own work levels (kMaxLevels + 1 histogram, cursor and level-start bins)
// and its own counters (kCtrClaim, kCtrItems, kCtrFirst).
constexpr int kTeamRobots = 8;
constexpr int kSmallSpheres = 256;
constexpr int kTeamSpheres = 512;
constexpr int kNumClasses = 3;
constexpr int kLevelBins = kNumClasses * (kMaxLevels + 1);
// BatchDev::counters: [0] queries handed to the full instance (entries of
// BatchDev::redo), [1] its claim counter, [2] abort flag; per class c the
// claim counter, the number of work items and the first sorted position of
// its queries
constexpr int kCtrRedo = 0;
constexpr int kCtrRedoClaim = 1;
constexpr int kCtrAbort = 2;
constexpr int kNumCounters = 16;
MRV_HD constexpr int kCtrClaim(int c) { return 4 + 3 * c; }
MRV_HD constexpr int kCtrItems(int c) { return 5 + 3 * c; }
MRV_HD constexpr int kCtrFirst(int c) { return 6 + 3 * c; }
static_assert(kCtrFirst(kNumClasses - 1) < kNumCounters, "counters fit");
// queries of point robots only with at most this many spheres check one
// state per lane (flavor A), in the team or large-team class
constexpr int kFlavorAMaxSpheres = 16;
// work class of a query with n robots and M spheres
MRV_HD constexpr int work_class(int n, int M) {
  return (n > kTeamRobots || M > kTeamSpheres) ? 2 : (M > kSmallSpheres ? 1 : 0);
}
constexpr int kNumStats = 16;         // statistics counters of a call (see mrv_stats)
// k_main's q_single for the pass of the full large-team instance over the
// queries the default instances handed over (BatchDev::redo)
constexpr int kRedoPass = -2;

// device error bits (BatchDev::err)
enum : uint32_t {
  kErrRobotId = 1u << 0,
  kErrEnvId = 1u << 1,
  kErrRobots = 1u << 2,      // 0 or > MRV_MAX_ROBOTS robots, or bad offsets
  kErrWaypoints = 1u << 3,   // bad waypoint offsets / counts
  kErrSteps = 1u << 4,       // negative steps or T > MRV_MAX_STEPS
  kErrSpheres = 1u << 5,     // > MRV_MAX_QUERY_SPHERES spheres in a query
  kErrDof = 1u << 6,         // wp_stride < dof
  kErrTimeout = 1u << 7,     // persistent kernel exceeded its clock budget
  kErrAbort = 1u << 8,       // abort flag observed
  kErrChecked = 1u << 9,     // MRV_CHECKED build: an index left its array
};

// The error record of a call: err[0] the bits above; in the MRV_CHECKED
// build err[1] = the first failing check site (below), err[2] its index and
// err[3] the extent it was checked against (low 32 bits each).
constexpr int kErrWords = 4;

// Index checks of the MRV_CHECKED build, one per array access class: a
// failing check records its site and redirects the access to element 0 of
// the same array (in bounds), so the kernel runs to its end without a fault
// and the call reports MRV_ERR_CUDA naming the site.
#define MRV_CHECK_SITES(X)                                                    \
  X(HIST, "k_prep: level-histogram bin")                                      \
  X(SEGSTEPS, "k_prep: waypoint step count index")                            \
  X(LEVELS, "k_levels: level-start entry")                                    \
  X(SCATTER, "k_scatter: sorted position")                                    \
  X(SORTED, "k_main: sorted query index")                                     \
  X(QUERY, "k_main: query index")                                             \
  X(FINISH_PAIR, "k_finish: robot pair decoded from the FFC key")             \
  X(SLOTS, "run_chunk: robot slot of the query")                              \
  X(PAIRTAB, "run_chunk: robot-pair table entry")                             \
  X(PAIRTAB_PREFIX, "run_chunk: frame-pair prefix (16 bits)")                 \
  X(CHAIN, "slice_b: FK chain slot in the link-frame buffer")                 \
  X(WAYPOINT, "interp: waypoint row")                                         \
  X(LINK, "frame index of a sphere or bounding sphere")                       \
  X(FRAME_SLOT, "frame slot (robot x frame) of a bounding sphere or mask")    \
  X(SPHERE, "sphere center of the query (P)")                                 \
  X(GRID_CELL, "obstacle grid cell")                                          \
  X(GRID_ITEM, "obstacle grid item")                                          \
  X(OBST_SPHERE, "obstacle sphere index")                                     \
  X(OBST_BOX, "obstacle box index")                                           \
  X(OBST_CYL, "obstacle cylinder index")                                      \
  X(SELF_GROUP, "self-pair group frames")                                     \
  X(SELF_BLOCK, "self-pair block rows / columns (10-bit offsets)")            \
  X(SELF_MASK, "self-pair block row mask")                                    \
  X(SELF_PAIR, "self-pair list entry")                                        \
  X(CAND, "candidate list entry")                                             \
  X(ROBOT_CULL, "large-team robot cull list")                                 \
  X(FLAVOR_A, "one-lane-per-state sphere buffer")                             \
  X(RECT, "self-pair rectangle rows / columns")                               \
  X(CLEAR_OUT, "k_clearance: output or sphere index")

enum : uint32_t {
  kCkNone = 0,
#define MRV_CK_ENUM(name, text) kCk_##name,
  MRV_CHECK_SITES(MRV_CK_ENUM)
#undef MRV_CK_ENUM
  kCkCount
};

struct alignas(16) ModelDev {
  // the FK parameters first, each row 16-byte aligned (read as float4)
  float base[12];                // base transform, 3x4 row-major
  float flange[12];              // flange transform, 3x4 row-major
  float dh[MRV_MAX_DOF][4];      // cos(alpha), sin(alpha), a, d
  float th0[MRV_MAX_DOF];        // theta_offset
  float link_bs[kMaxLinks][4];   // frame-local bounding sphere (radius < 0: empty)
  int32_t kind, dof, n_spheres, n_self;
  int32_t live;
  float point_z;
  float r2max;                   // largest squared sphere radius
  const float4 *spheres;         // local xyz, radius; sorted by frame
  const int32_t *sphere_link;
  const uint32_t *self_pairs;    // x | y << 16 with x < y, grouped by frame
                                 // pair, padded by repeating the last pair to a
                                 // multiple of 4 (indices of the sorted spheres)
  const int4 *self_rects;        // the same pairs as rectangles (x0, x1, y0, y1):
                                 // rows x0..x1-1 against columns y0..y1-1
  int32_t n_rects;               // 0: use the sparse list
  int32_t n_links;               // frames 0..n_links-1 (DH: dof + 2, point: 2)
  int32_t link_start[kMaxLinks + 1];  // spheres (sorted by frame) of frame l
  const int4 *self_groups;       // (frame u, frame v, first pair, count)
  const int4 *self_blocks;       // per group: first row sphere, first column
                                 // sphere, rows | columns << 16 (columns <= 32),
                                 // first row mask; null: pair list only
  const uint32_t *self_masks;    // per block row: bit c = pair with column c
  int32_t n_groups;
  int32_t n_masks;               // self-pair block rows (entries of self_masks)
  uint32_t frame_mask;           // bit l: frame l holds spheres
  const int32_t *perm;           // sorted sphere index -> caller's index
};
static_assert(offsetof(ModelDev, base) % 16 == 0 && offsetof(ModelDev, flange) % 16 == 0 &&
                  offsetof(ModelDev, dh) % 16 == 0 && offsetof(ModelDev, link_bs) % 16 == 0 &&
                  sizeof(ModelDev) % 16 == 0,
              "FK rows of a model are read as float4");

struct EnvDev {
  int32_t n_spheres, n_aabbs;
  int32_t live;
  float c2max;                   // largest |center|^2 of the obstacle spheres
  float r2max;                   // largest squared obstacle radius
  int32_t pad[3];
  const float4 *spheres;         // world xyz, radius
  const float *sphere_k;         // |center|^2 - radius^2 per obstacle sphere
  const float4 *box_lo;          // n_aabbs: lo xyz (w unused)
  const float4 *box_hi;          // n_aabbs: hi xyz (w unused)
  // uniform grid over the obstacles for frame bounding spheres of radius
  // <= g_R (g_R < 0: none): cell (ix, iy, iz) of a center x is
  // floor((x - g_lo) * g_inv_h) per axis; outside 0..g_dims-1 it overlaps no
  // obstacle.  Cell c = (iz * g_dims[1] + iy) * g_dims[0] + ix lists its
  // obstacle spheres, boxes and cylinders (counts in g_cnt) at
  // g_items[g_off[c] .. g_off[c+1]).
  float g_lo[3], g_inv_h, g_R;
  int32_t g_dims[3];
  const int32_t *g_off;
  const uint32_t *g_cnt;         // per cell: spheres | boxes << 16 (cylinders follow)
  const uint16_t *g_items;
  // solid cylinders with flat caps
  int32_t n_cyl;
  int32_t g_nitems;              // entries of g_items
  const float4 *cyl_a;           // axis end a xyz, radius
  const float4 *cyl_u;           // unit axis (a -> b) xyz, length |b - a|
};

// per-query derived record (written by the preparation kernel)
struct QueryDev {
  int32_t T;          // composite step count (states 0..T)
  int32_t n;          // robots
  int32_t M;          // spheres summed over robots
  int32_t ntiles;     // 32-state tiles
  int32_t split;      // slices per tile
  int32_t spt;        // states per slice (32 / split)
  int32_t nslices;    // slices per phase (ntiles * split)
  int32_t nphase;     // 2 for hierarchical MV (env pass, then pair pass) and for
                      // pairs-first MV (adjacent pairs, then the rest), else 1
  int32_t nchunks;    // work items of this query
  int32_t cte;        // slices per work item
  int32_t env;        // env slot or -1
  uint32_t bits;      // bit 0: FFC, bit 1: flavor A (lane = state), bit 2: invalid,
                      // bits 3-4: work class (work_class)
  float rho2;         // largest squared sphere radius of the query's robots
  int32_t nadj;       // pairs-first MV: adjacent robot pairs (0: the order is off)
  int32_t nchain;     // robots that are kinematic chains (one FK chain per state each)
  int32_t njoint;     // joints summed over those robots
  uint32_t adj[4];    // pairs-first MV: bit p = pair p (in (i, j) order) is adjacent
  long long adjtests;   // pairs-first MV: sphere tests per state of the adjacent pairs
  long long pairtests;  // robot-robot sphere tests per state
  long long envtests;   // robot-obstacle sphere + self tests per state (MV with env)
  long long boxtests;   // robot-box tests per state (MV with env)
  long long cyltests;   // robot-cylinder tests per state (MV with env)
};

struct BatchDev {
  int32_t n_queries, n_slots, n_waypoints, wp_stride;
  uint32_t flags;
  float resolution;
  int32_t default_env;               // env slot or -1
  int32_t pad0;
  const int32_t *q_robot_off;
  const int32_t *slot_robot_id;
  const int32_t *slot_wp_off;
  const float *waypoints;
  const int32_t *seg_steps;          // may be null (start/goal form)
  const int32_t *q_env_id;           // may be null
  const uint8_t *q_kind;             // may be null (all MV unless forced)
  int32_t forced_kind;               // -1 = q_kind, else MRV_KIND_*
  int32_t slices_per_item;
  int32_t tile_split;
  int32_t mv_order;                  // tuning: 1 = hierarchical order for MV batches naming none
  // derived (device scratch)
  int32_t *slot_tau;                 // n_waypoints: time of each waypoint
  QueryDev *q;                       // n_queries
  int32_t *q_hit;                    // MV: 1 once a collision is found
  int32_t *q_best;                   // FFC: min key t << 7 | pair index
  float *q_minclr;                   // exhaustive MV: min clearance (as ordered int)
  int32_t *sorted;                   // queries by class, nchunks (desc), then FFC before MV
  int32_t *hist;                     // kLevelBins bins (class 0, 1, then 2)
  int32_t *level_start;              // kLevelBins
  int32_t *cursor;                   // 2 x kLevelBins: each bin's next FFC and next MV position
  int32_t *redo_flag;                // n_queries: 1 once the query is listed in redo
  int32_t *q_states;                 // n_queries: states the default instances counted
  int32_t *redo;                     // n_queries: queries whose checks need a path the
                                     // default instances do not have (candidate lists
                                     // overflowing, self pairs without blocks), rerun
                                     // whole by the full large-team instance
  int32_t *counters;                 // kNumCounters: the abort flag and per-class claim
                                     // counter, items and first sorted position (kCtr*)
  uint32_t *err;                     // kErrWords: error bits, check site, index, extent
  unsigned long long *stats;         // [0] states checked, [1] tests executed,
                                     // [2] states available, [3] tests available,
                                     // [4] items, [5] box tests executed,
                                     // [6] FK chains, [7] spheres placed,
                                     // [8] cylinder tests executed; the
                                     // method's dense work of the states
                                     // checked: [9] sphere-sphere tests
                                     // (robot-robot, obstacle spheres, self
                                     // pairs), [10] box tests, [11] cylinder
                                     // tests, [12] joints, [13] chains,
                                     // [14] sphere placements, [15] queries
                                     // rerun by the full instance
  // tables
  const ModelDev *models;
  int32_t n_models;
  const EnvDev *envs;
  int32_t n_envs;
  long long clock_budget;            // persistent kernel: clock64 ticks (0 = none)
  int32_t classes;                   // host: bit c = the batch may hold class-c queries (launch its kernel)
  int32_t full;                      // the run uses the full instances of the persistent kernel
                                     // (minimum clearance, MRV_NO_BROADPHASE): dense path, flavor A
  int32_t clr;                       // exhaustive MV reports each query's minimum clearance
  int32_t pad1;
};

}  // namespace mrv
