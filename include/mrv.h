/*
 * mrv.h — multi-robot motion validation on GB300 (sm_103a): C ABI.
 *
 * Two primitives over synchronized multi-robot motions (paper Sec. III):
 *   MotionValidation  (MV,  Alg. 1): boolean validity with early termination
 *                     on any robot-obstacle, self or robot-robot collision;
 *   FindFirstConflict (FFC, Alg. 2): the earliest robot-robot conflict
 *                     (timestep, robot i, robot j).
 * Robots are kinematic chains (modified DH) or point robots, approximated by
 * spheres (Sec. II-B); obstacles are spheres, axis-aligned boxes ("simple
 * geometries", Sec. III-A) and solid cylinders (the Cage obstacles, Sec. V-A);
 * motions are start/goal pairs discretised at a C-space resolution
 * (Sec. IV-A3) or timed waypoint paths; shorter paths are padded with their
 * last configuration (Sec. III-A).  MV also comes in the prioritized
 * planner's form (one robot against higher-priority paths, Sec. IV-C).
 *
 * Conventions for every entry point:
 *   - return value: MRV_OK (0) or a negative MRV_ERR_* code; no call aborts
 *     the process.  mrv_last_error() returns a message for the calling thread.
 *   - the caller owns every input and output buffer; uploads copy into
 *     device memory owned by the context.
 *   - pointers are host pointers unless the batch has MRV_PTRS_ON_DEVICE set,
 *     in which case every input array of the batch and every output array of
 *     the call are device pointers on the context's device.
 *   - work runs on the context's CUDA stream; a call returns after its
 *     outputs are written unless MRV_ASYNC is set (then mrv_sync() waits and
 *     reports device-side errors).  MRV_ASYNC requires MRV_PTRS_ON_DEVICE.
 *   - robot indices (i, j) in a conflict are 0-based slot positions inside
 *     the query (the paper numbers robots from 1).
 */
#ifndef MRV_H
#define MRV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MRV_OK 0
#define MRV_ERR_ARG (-1)       /* malformed argument or batch               */
#define MRV_ERR_OOM (-2)       /* device or host allocation failed          */
#define MRV_ERR_NOT_FOUND (-3) /* unknown or released robot / env id        */
#define MRV_ERR_CUDA (-4)      /* CUDA runtime error                        */
#define MRV_ERR_TIMEOUT (-5)   /* a bounded device or host wait ran out     */
#define MRV_ERR_BUSY (-6)      /* admission refused / queue full            */
#define MRV_ERR_LIMIT (-7)     /* a size beyond a documented maximum        */

/* ---- limits ------------------------------------------------------------ */
/* Queries of up to 8 robots run on the small-team kernel layout (up to 256
 * spheres) or the team layout (up to 512); larger ones (the 16-arm Cage team
 * of Sec. V-A) on a large-team layout; the team and large-team instances are
 * launched beside the first when a batch may hold such queries (always for
 * MRV_PTRS_ON_DEVICE batches). */
#define MRV_MAX_ROBOTS 16          /* robots per query (120 pairs)          */
#define MRV_MAX_DOF 8              /* joints per robot                      */
#define MRV_MAX_SPHERES 256        /* spheres per robot model               */
#define MRV_MAX_QUERY_SPHERES 1024 /* spheres summed over a query's robots  */
#define MRV_MAX_STEPS ((1 << 24) - 1) /* composite step count T of a query  */

/* ---- robot kinds ------------------------------------------------------- */
#define MRV_ROBOT_DH_CHAIN 0
#define MRV_ROBOT_POINT 1

/* ---- batch flags ------------------------------------------------------- */
#define MRV_CHECK_ENV 0x1u        /* robot-obstacle + self checks (Alg. 1)  */
#define MRV_HIERARCHICAL 0x2u     /* Alg. 1 hierarchical order (MV)         */
#define MRV_EXHAUSTIVE 0x4u       /* no early termination (Sec. IV-A1)      */
#define MRV_PTRS_ON_DEVICE 0x8u   /* inputs and outputs are device pointers */
#define MRV_ASYNC 0x10u           /* return before completion (see above)   */
#define MRV_PER_QUERY_LAUNCH 0x20u /* baseline: one synchronous kernel
                                      launch per query                      */
#define MRV_NO_BROADPHASE 0x40u   /* test every sphere pair (no frame-level
                                     bounding-sphere culling); same results */
#define MRV_PRIORITY 0x100u       /* MV of prioritized planning (PP-ST-RRT,
                                     Sec. IV-C): slot 0 of each MV query is
                                     the robot being planned, slots 1..n-1
                                     robots of higher priority whose paths
                                     act as moving obstacles.  The obstacle
                                     and self checks run for slot 0 only and
                                     the robot-robot checks for the pairs
                                     (0, j) only.  FFC queries ignore it.   */
#define MRV_LINEAR 0x80u          /* MV visits the states of a tile in the
                                     linear order t = 32 b + l (the map FFC
                                     uses, Sec. IV-B) instead of the rake
                                     order t = b + nb l of Alg. 1 / Fig. 2;
                                     same verdicts, different effort        */
#define MRV_PAIRS_FIRST 0x200u    /* MV checks the robot pairs likely to
                                     collide first, the mixed strategy of
                                     Sec. III-A: adjacent fixed-base robots
                                     (kinematic chains whose bases are within
                                     1.25x of either one's nearest other
                                     fixed base).  Each slice runs twice:
                                     those pairs, then the obstacle and self
                                     checks and the other pairs.  Same
                                     verdicts, different effort.  Queries
                                     without such a pair run the combined
                                     order; FFC queries and MRV_EXHAUSTIVE
                                     runs ignore it; not with
                                     MRV_HIERARCHICAL or MRV_PRIORITY.      */

/* ---- query kinds (mrv_run) ---------------------------------------------- */
#define MRV_KIND_MV 0
#define MRV_KIND_FFC 1

typedef struct mrv_ctx mrv_ctx;

/* Creates a context on CUDA device `device`; work is issued on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out is owned by the
 * caller and freed with mrv_destroy.  MRV_ERR_CUDA when the device is absent. */
int mrv_create(mrv_ctx **out, int device, void *cuda_stream);
int mrv_destroy(mrv_ctx *ctx);
/* Message of the last failing call on this thread (never NULL; owned by the
 * library, valid until the next call on this thread). */
const char *mrv_last_error(mrv_ctx *ctx);
/* Changes the stream later calls are issued on. */
int mrv_set_stream(mrv_ctx *ctx, void *cuda_stream);

/* ---- robot models (Sec. II-B: kinematic chain + spheres) ---------------- */
typedef struct {
  int32_t kind;             /* MRV_ROBOT_DH_CHAIN or MRV_ROBOT_POINT          */
  int32_t dof;              /* DH: 1..MRV_MAX_DOF; POINT: 2 (x, y at point_z)
                               or 3 (x, y, z)                                 */
  const float *dh;          /* DH: dof x 4 row-major (a, alpha, d, theta_off);
                               joint k maps frame k-1 to frame k by
                               RotX(alpha) TransX(a) RotZ(theta_off+q_k)
                               TransZ(d) (Craig's modified DH)                */
  const float *flange;      /* DH: 3x4 fixed transform after the last joint
                               (frame dof+1); NULL = identity                 */
  const float *base;        /* 3x4 row-major world <- base transform; NULL =
                               identity                                       */
  float point_z;            /* POINT with dof 2: fixed z                      */
  int32_t n_spheres;        /* 1..MRV_MAX_SPHERES                             */
  const int32_t *sphere_link; /* n_spheres: 0 = base frame, k = frame after
                               joint k, dof+1 = flange frame (DH); POINT: 0 =
                               base, 1 = moving frame                         */
  const float *sphere_xyzr; /* n_spheres x 4: link-local center, radius > 0   */
  int32_t n_self_pairs;     /* self-collision pairs checked with the env      */
  const int32_t *self_pairs; /* n_self_pairs x 2 sphere indices, or NULL      */
} mrv_robot_desc;

/* Copies a robot model (host pointers) to the device.  *robot_id_out is the
 * handle used in batches.  MRV_ERR_ARG / MRV_ERR_LIMIT on malformed models. */
int robot_model_upload(mrv_ctx *ctx, const mrv_robot_desc *desc, int32_t *robot_id_out);

/* ---- environments (obstacle set E, Alg. 1) ------------------------------ */
typedef struct {
  int32_t n_spheres;
  const float *spheres_xyzr;  /* n_spheres x 4, world frame                  */
  int32_t n_aabbs;
  const float *aabb_lohi;     /* n_aabbs x 6: lo x,y,z then hi x,y,z         */
  int32_t n_cylinders;        /* solid cylinders with flat caps (the Cage
                                 obstacles of Sec. V-A); may be 0            */
  const float *cylinders;     /* n_cylinders x 7: axis end a x,y,z, axis end
                                 b x,y,z, radius; |b - a| > 0, radius >= 0.
                                 A sphere collides with a cylinder when its
                                 center is closer to the solid than its
                                 radius (distance 0 inside)                */
} mrv_env_desc;

/* Copies an obstacle set (host pointers) to the device.  MRV_ERR_ARG on a
 * NULL array with a non-zero count, a non-finite value, a negative radius,
 * a box with lo > hi or a cylinder whose axis ends coincide. */
int env_upload(mrv_ctx *ctx, const mrv_env_desc *desc, int32_t *env_id_out);
/* Drops the upload's reference (robots and envs share the id space); the
 * device memory is freed once no call in flight uses it (the context's
 * stream is synchronized first). */
int mrv_release(mrv_ctx *ctx, int32_t id);

/* ---- batches of queries --------------------------------------------------
 * A ragged CSR batch.  Query q has slots q_robot_off[q] .. q_robot_off[q+1]-1
 * (1..MRV_MAX_ROBOTS robots; slot order defines robot indices i, j).  Slot s
 * uses robot model slot_robot_id[s] and waypoints slot_wp_off[s] ..
 * slot_wp_off[s+1]-1; waypoint w is the row waypoints[w*wp_stride ..] whose
 * first dof entries are the configuration.
 *   - timed form (seg_steps != NULL): seg_steps[w] >= 1 interpolation steps
 *     from waypoint w to the next one of its slot (ignored for a slot's last
 *     waypoint); slot times start at 0; a slot past its end holds its last
 *     configuration (padding, Sec. III-A).
 *   - start/goal form (seg_steps == NULL): every slot has exactly 2
 *     waypoints; each robot needs ceil(|g - s|_2 / resolution) steps (0 if it
 *     does not move) and the composite motion takes the maximum T over its
 *     robots, all robots time-scaled to start and finish together
 *     (Sec. IV-A3).  T is computed in IEEE double, operations separately
 *     rounded, summing squared joint differences in joint order.
 * States t = 0..T (T+1 states) are checked; T <= MRV_MAX_STEPS. */
typedef struct {
  int32_t n_queries;
  int32_t n_slots;           /* = q_robot_off[n_queries]                     */
  int32_t n_waypoints;       /* = slot_wp_off[n_slots]                       */
  int32_t env_id;            /* obstacle set of every query; -1 = none       */
  const int32_t *q_robot_off;   /* n_queries + 1                             */
  const int32_t *slot_robot_id; /* n_slots                                   */
  const int32_t *slot_wp_off;   /* n_slots + 1                               */
  const float *waypoints;       /* n_waypoints x wp_stride                   */
  int32_t wp_stride;            /* >= the largest dof used                   */
  const int32_t *seg_steps;     /* n_waypoints, or NULL (start/goal form)    */
  float resolution;             /* start/goal form: C-space units per step   */
  const int32_t *q_env_id;      /* n_queries env ids (-1 none) or NULL       */
  const uint8_t *q_kind;        /* n_queries MRV_KIND_* (mrv_run) or NULL    */
  uint32_t flags;               /* MRV_* batch flags                         */
} mrv_batch;

/* conflict record (Alg. 2): {-1,-1,-1} = none */
typedef struct {
  int32_t t, i, j;
} mrv_conflict;

/* MotionValidation (Alg. 1) of every query: valid_out[q] = 1 iff no state
 * t in 0..T has a robot-robot collision or (MRV_CHECK_ENV) a robot-obstacle
 * or self collision.  Early termination per query unless MRV_EXHAUSTIVE.
 * min_clearance_out (nullable; requires MRV_EXHAUSTIVE): signed minimum
 * clearance over every check of the query, +inf when no check applies. */
int mv_validate(mrv_ctx *ctx, const mrv_batch *batch, uint8_t *valid_out, float *min_clearance_out);

/* FindFirstConflict (Alg. 2) of every query: the lexicographically smallest
 * (t, i, j) with robots i < j overlapping at state t.  No obstacle or self
 * checks (Sec. III-B). */
int ffc_find(mrv_ctx *ctx, const mrv_batch *batch, mrv_conflict *out);

/* Mixed batch in one persistent launch: query q is MV when q_kind[q] ==
 * MRV_KIND_MV (valid_out[q] written) and FFC otherwise (conflict_out[q]
 * written); entries of the other output are left untouched. */
int mrv_run(mrv_ctx *ctx, const mrv_batch *batch, uint8_t *valid_out, mrv_conflict *conflict_out);

/* ---- MotionValidation without allocation ---------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory while they validate motions, e.g. a planner
 * inside a latency-bounded control loop (cudaMalloc / cudaFree can block, and
 * cudaFree synchronizes the device) or an application whose device memory is
 * already fully budgeted by its own allocator.  It computes exactly what
 * mv_validate computes (early termination, MRV_CHECK_ENV honoured), but its
 * per-call scratch is one static device array of about 0.84 MB that every GPU
 * loading the library holds until the process exits, so the call performs no
 * allocation.  The caller passes device pointers (MRV_PTRS_ON_DEVICE) for the
 * batch and valid_out; at most MRV_NOALLOC_MAX_QUERIES queries and
 * MRV_NOALLOC_MAX_WAYPOINTS waypoints (MRV_ERR_LIMIT beyond); MRV_ASYNC,
 * MRV_EXHAUSTIVE and MRV_PER_QUERY_LAUNCH are rejected (MRV_ERR_ARG).  The
 * array's device address is looked up on every call (the lookup allocates
 * nothing).  The call waits for its result, so it must not be called while
 * the context's stream is being captured into a CUDA graph (MRV_ERR_ARG).
 * All calls on a device share the array: each call resets what must start
 * from zero, and calls whose work overlaps on the device race, so issue them
 * on one stream or synchronize between them.  Returns after valid_out is
 * written; mrv_get_stats then describes this call. */
#define MRV_NOALLOC_MAX_QUERIES 4096
#define MRV_NOALLOC_MAX_WAYPOINTS 65536
int mv_validate_noalloc(mrv_ctx *ctx, const mrv_batch *batch, uint8_t *valid_out);

/* Diagnostic: per-sphere minimum clearance of query `q` of the batch at the
 * listed timesteps (0 <= ts[k] <= T).  out: nt x M floats, M = spheres of the
 * query's robots in slot order; each value is the minimum over the checks
 * that involve the sphere (other robots' spheres; obstacles and self pairs
 * when MRV_CHECK_ENV), +inf when none.  Pointer kinds follow the batch
 * flag; MRV_PRIORITY does not restrict it (every robot and pair is
 * reported). */
int mrv_clearance(mrv_ctx *ctx, const mrv_batch *batch, int32_t q, const int32_t *ts, int32_t nt,
                  float *out);

/* Waits for MRV_ASYNC work on the context's stream; returns its status. */
int mrv_sync(mrv_ctx *ctx);

/* ---- failure detection -----------------------------------------------------
 * kernel_budget_ms > 0 bounds the persistent kernel of every later call:
 * each warp stops taking work items once its SM clock has run that long
 * since the warp started, and the call returns MRV_ERR_TIMEOUT (its outputs
 * are then incomplete).  0 = no bound (default).  The kernel never waits on
 * anything, so the bound only cuts long batches short; the context stays
 * usable.  (No counterpart in the paper.) */
typedef struct {
  double kernel_budget_ms;
} mrv_limits;
int mrv_set_limits(mrv_ctx *ctx, const mrv_limits *limits);

/* ---- statistics of the last completed call -------------------------------- */
typedef struct {
  uint64_t states_available; /* sum over queries of (T+1)                    */
  uint64_t states_checked;   /* states whose checks ran                      */
  uint64_t sphere_tests;     /* sphere-sphere + sphere-box tests executed,
                                including frame bounding-sphere tests        */
  uint64_t sphere_tests_available; /* tests of an exhaustive run             */
  uint64_t work_items;       /* persistent-scheduler items                   */
  int32_t n_valid, n_conflicts;
  float device_ms;           /* kernel time of the last call (CUDA events)   */
  uint64_t box_tests;        /* the sphere-box part of sphere_tests           */
  uint64_t fk_chains;        /* (state, robot) kinematic chains evaluated     */
  uint64_t spheres_placed;   /* sphere centers computed (states x spheres)    */
  uint64_t cylinder_tests;   /* the sphere-cylinder part of sphere_tests      */
  /* The method's own work on the states checked (each state once): what a
   * dense check of those states performs, whatever the broadphase skipped.
   * It is the numerator of the FP32 roofline of a call. */
  uint64_t method_sphere_tests;   /* robot-robot, obstacle-sphere and self
                                     sphere pairs                             */
  uint64_t method_box_tests;      /* sphere-box pairs                         */
  uint64_t method_cylinder_tests; /* sphere-cylinder pairs                    */
  uint64_t method_joints;         /* joints of the kinematic-chain robots     */
  uint64_t method_chains;         /* kinematic chains (one per robot, state)  */
  uint64_t method_spheres;        /* sphere placements                        */
  /* Queries the default kernel instance handed to the full one: a state
   * whose broadphase candidate lists overflowed, or self pairs of a model
   * without row blocks.  The full instance reruns every work item of such a
   * query; states_checked and the method_* counters count each state once,
   * the executed-work counters (sphere_tests, fk_chains, spheres_placed, ...)
   * both runs. */
  uint64_t queries_redone;
} mrv_stats;
int mrv_get_stats(mrv_ctx *ctx, mrv_stats *out);

/* ---- scheduling knobs (persistent work-stealing kernel) ------------------
 * Work is cut into slices: a 32-state tile of a query split into tile_split
 * slices (MV: rake lanes l = p, p+split, ...; FFC: consecutive states); a
 * work item is slices_per_item consecutive slices of one query. */
typedef struct {
  int32_t slices_per_item;   /* slices per work item (>= 1)                  */
  int32_t warps_per_block;   /* 1..12, blocks of the small-team and team
                                instances (queries of up to 256 / 512
                                spheres: 13 / 17.3 KB of shared memory per
                                warp, up to 16 / 12 warps per SM); the
                                large-team instance uses 6 warps of 34.8 KB */
  int32_t blocks_per_sm;     /* 0 = as many as fit                           */
  int32_t tile_split;        /* 1, 2, 4, 8, 16 or 32 slices per 32-state tile for
                                kinematic-chain queries (point-robot queries
                                always use whole tiles)                      */
  int32_t mv_order;          /* order of MV queries with obstacle checks in
                                early-exit batches whose flags name none
                                (MRV_HIERARCHICAL, MRV_PAIRS_FIRST): 0 the
                                combined order, 1 the hierarchical order
                                (MRV_EXHAUSTIVE runs use the combined one).
                                Same verdicts; mrv_autotune times both.     */
} mrv_tuning;
int mrv_set_tuning(mrv_ctx *ctx, const mrv_tuning *t);
int mrv_get_tuning(mrv_ctx *ctx, mrv_tuning *t);

/* Times candidate tunings on `batch` (MRV_PTRS_ON_DEVICE, run through
 * mrv_run semantics): 1, 2 or 4 slices per item x 2, 4, 8 or 16 slices per
 * tile x 4- or 8-warp blocks, and both MV orders when the batch has obstacle
 * checks and names no order; each scored by the fastest of four timed runs
 * (twelve when a run takes under 2 ms).
 * Keeps the fastest in the context and caches it in the text file
 * `cache_path` (nullable) keyed by device name and a batch class (robot
 * count, sphere count and length buckets, query kinds).  A cached entry is
 * reused without timing. */
int mrv_autotune(mrv_ctx *ctx, const mrv_batch *batch, const char *cache_path, mrv_tuning *chosen);

/* ---- CUDA-graph replay of one batch ----------------------------------------
 * Captures the whole mixed run of a device-resident batch (counter reset,
 * preparation kernels, both persistent kernel instances, result kernel) into a CUDA graph
 * bound to these exact pointers; mrv_graph_launch replays it on the
 * context's stream (asynchronous; mrv_sync waits). */
typedef struct mrv_graph mrv_graph;
int mrv_graph_create(mrv_ctx *ctx, const mrv_batch *batch, uint8_t *valid_out, mrv_conflict *conflict_out,
                     mrv_graph **out);
int mrv_graph_launch(mrv_graph *g);
int mrv_graph_destroy(mrv_graph *g);

/* ---- serving: continuous batching over streams ------------------------------
 * A server owns `n_streams` CUDA streams and a scheduler thread.  Requests
 * (host batches) are copied at submission; the scheduler admits waiting
 * requests in arrival order whenever a stream is free and the request's
 * device footprint fits in the free part of `device_budget_bytes`, packs
 * every admitted request into one micro-batch, and runs it while other
 * micro-batches are still on the device.  Robot and env ids refer to the
 * context's resident uploads.  At creation every stream's device arena and
 * pinned staging are sized for a micro-batch of max_batch_queries queries
 * of up to 8 robots on two waypoints each (halved until all of them take at
 * most half of the device's free memory), micro-batches are packed within
 * those buffers, and only a single request larger than them makes its
 * stream's buffers grow.  The budget is clamped to the device's free memory
 * after that sizing plus the arenas themselves (see mrv_server_stats). */
typedef struct mrv_server mrv_server;
typedef struct {
  int32_t n_streams;            /* concurrent micro-batches (1..16)          */
  size_t device_budget_bytes;   /* admission limit on device footprint       */
  int32_t max_batch_queries;    /* queries per micro-batch                   */
  int32_t max_pending;          /* waiting requests before MRV_ERR_BUSY      */
} mrv_server_opts;
int mrv_server_create(mrv_ctx *ctx, const mrv_server_opts *opts, mrv_server **out);
int mrv_server_destroy(mrv_server *s);
/* Copies the host batch (flags: MRV_CHECK_ENV, MRV_EXHAUSTIVE only) and
 * queues it; *ticket identifies the request. */
int mrv_server_submit(mrv_server *s, const mrv_batch *batch, uint64_t *ticket);
/* Waits up to timeout_ms for the request, then copies its results (host
 * pointers, n_queries entries; either may be NULL) and forgets the ticket.
 * MRV_ERR_TIMEOUT leaves the request pending. */
int mrv_server_wait(mrv_server *s, uint64_t ticket, int32_t timeout_ms, uint8_t *valid_out,
                    mrv_conflict *conflict_out);
typedef struct {
  uint64_t submitted, completed, rejected, micro_batches, queries;
  uint64_t max_inflight;        /* largest number of micro-batches in flight */
  double busy_ms;               /* device time summed over micro-batches     */
  uint64_t device_budget_bytes; /* admission budget in force (after clamping) */
  uint64_t device_free_bytes;   /* device free memory after the buffers were
                                   sized at creation                        */
  uint64_t presized_queries;    /* queries per micro-batch the buffers hold  */
} mrv_server_stats;
int mrv_server_get_stats(mrv_server *s, mrv_server_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* MRV_H */
