// Host runtime of the C ABI declared in include/mrv.h: contexts, the
// device-resident model / environment registry, batch staging, the launch
// sequence (prepare -> persistent kernel -> results), CUDA-graph capture and
// statistics.  Every entry point returns a status code; nothing aborts.
#include "mrv_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <mutex>
#include <utility>

namespace mrv {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Host-side fault injection for tests: whenever the environment variable
// MRV_FAULT_INJECT_ALLOC takes a value not seen before, the next device
// allocation of this process fails as if the device were out of memory.
cudaError_t dev_malloc(void **p, size_t n) {
  static std::mutex mu;
  static std::string seen;
  {
    std::lock_guard<std::mutex> lk(mu);
    const char *v = std::getenv("MRV_FAULT_INJECT_ALLOC");
    if (v && *v && seen != v) {
      seen = v;
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(p, n);
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? MRV_ERR_OOM : MRV_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// scratch arena
// ---------------------------------------------------------------------------

static size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// The arena's layout, one walk for both sizing (p == nullptr) and carving:
// every array starts on a 256-byte boundary.  Returns the bytes it spans.
size_t Scratch::layout(int64_t nq, int64_t ns, int64_t nw, int64_t stride, char *p) {
  size_t o = 0;
  auto take = [&](size_t n) {
    o = align_up(o, 256);
    void *r = p ? p + o : nullptr;
    o += n;
    return r;
  };
  auto set = [&](auto **dst, size_t n) {
    void *r = take(n);
    if (p) *dst = static_cast<std::remove_pointer_t<decltype(dst)>>(r);
  };
  set(&slot_tau, sizeof(int32_t) * nw);
  set(&q, sizeof(QueryDev) * nq);
  set(&q_hit, sizeof(int32_t) * nq);
  set(&q_best, sizeof(int32_t) * nq);
  set(&q_minclr, sizeof(float) * nq);
  set(&sorted, sizeof(int32_t) * nq);
  set(&redo_flag, sizeof(int32_t) * nq);
  set(&redo, sizeof(int32_t) * nq);
  set(&q_states, sizeof(int32_t) * nq);
  set(&hist, sizeof(int32_t) * kLevelBins);
  set(&level_start, sizeof(int32_t) * kLevelBins);
  set(&cursor, sizeof(int32_t) * 2 * kLevelBins);
  set(&counters, sizeof(int32_t) * kNumCounters);
  set(&err, sizeof(uint32_t) * kErrWords);
  set(&stats, sizeof(unsigned long long) * kNumStats);
  set(&counts, sizeof(int32_t) * 4);
  // staged inputs
  set(&in_q_off, sizeof(int32_t) * (nq + 1));
  set(&in_slot_robot, sizeof(int32_t) * ns);
  set(&in_slot_wp, sizeof(int32_t) * (ns + 1));
  set(&in_wp, sizeof(float) * nw * stride);
  set(&in_steps, sizeof(int32_t) * nw);
  set(&in_q_env, sizeof(int32_t) * nq);
  set(&in_q_kind, sizeof(uint8_t) * nq);
  // staged outputs
  set(&out_valid, sizeof(uint8_t) * nq);
  set(&out_minclr, sizeof(float) * nq);
  set(&out_conf, sizeof(mrv_conflict) * nq);
  return align_up(o, 256);
}

size_t Scratch::bytes_for(int64_t nq, int64_t ns, int64_t nw, int64_t stride) {
  Scratch probe;
  return probe.layout(nq, ns, nw, stride, nullptr);
}

int Scratch::ensure(int64_t nq, int64_t ns, int64_t nw, int64_t stride, cudaStream_t st) {
  const size_t need = bytes_for(nq, ns, nw, stride);
  if (need > cap) {
    if (base) {
      cudaStreamSynchronize(st);
      cudaFree(base);
      base = nullptr;
      cap = 0;
    }
    size_t want = need + need / 4;
    cudaError_t e = dev_malloc(&base, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      return cuda_fail(e, "scratch allocation");
    }
    cap = want;
  }
  layout(nq, ns, nw, stride, static_cast<char *>(base));
  return MRV_OK;
}

void Scratch::release() {
  if (base) cudaFree(base);
  base = nullptr;
  cap = 0;
}

// ---------------------------------------------------------------------------
// batch launch
// ---------------------------------------------------------------------------

int validate_batch(mrv_ctx *ctx, const mrv_batch *b) {
  if (!b) return fail(MRV_ERR_ARG, "batch is NULL");
  if (b->n_queries < 0 || b->n_slots < 0 || b->n_waypoints < 0)
    return fail(MRV_ERR_ARG, "negative batch sizes");
  if (b->n_queries == 0) return MRV_OK;
  if (b->wp_stride < 1 || b->wp_stride > 64) return fail(MRV_ERR_ARG, "wp_stride %d outside 1..64", b->wp_stride);
  if (!b->q_robot_off || !b->slot_robot_id || !b->slot_wp_off || !b->waypoints)
    return fail(MRV_ERR_ARG, "missing batch array");
  if (b->flags & ~(uint32_t)(MRV_CHECK_ENV | MRV_HIERARCHICAL | MRV_EXHAUSTIVE | MRV_PTRS_ON_DEVICE | MRV_ASYNC |
                             MRV_PER_QUERY_LAUNCH | MRV_NO_BROADPHASE | MRV_LINEAR |
                             MRV_PRIORITY | MRV_PAIRS_FIRST))
    return fail(MRV_ERR_ARG, "unknown flag bits 0x%x", b->flags);
  if ((b->flags & MRV_PAIRS_FIRST) && (b->flags & (MRV_HIERARCHICAL | MRV_PRIORITY)))
    return fail(MRV_ERR_ARG, "MRV_PAIRS_FIRST excludes MRV_HIERARCHICAL and MRV_PRIORITY");
  if ((b->flags & MRV_ASYNC) && !(b->flags & MRV_PTRS_ON_DEVICE))
    return fail(MRV_ERR_ARG, "MRV_ASYNC requires MRV_PTRS_ON_DEVICE");
  if (!b->seg_steps && !(std::isfinite(b->resolution) && b->resolution > 0.f))
    return fail(MRV_ERR_ARG, "start/goal form needs a positive finite resolution");
  if (b->env_id != -1 && ctx->env_slot(b->env_id) < 0)
    return fail(MRV_ERR_NOT_FOUND, "unknown env id %d", b->env_id);
  if (!(b->flags & MRV_PTRS_ON_DEVICE)) {
    if (b->q_robot_off[0] != 0 || b->q_robot_off[b->n_queries] != b->n_slots)
      return fail(MRV_ERR_ARG, "q_robot_off must run from 0 to n_slots");
    if (b->slot_wp_off[0] != 0 || b->slot_wp_off[b->n_slots] != b->n_waypoints)
      return fail(MRV_ERR_ARG, "slot_wp_off must run from 0 to n_waypoints");
    for (int q = 0; q < b->n_queries; ++q) {
      const int n = b->q_robot_off[q + 1] - b->q_robot_off[q];
      if (n < 1) return fail(MRV_ERR_ARG, "query %d has no robot", q);
      if (n > MRV_MAX_ROBOTS) return fail(MRV_ERR_LIMIT, "query %d has %d robots (max %d)", q, n, MRV_MAX_ROBOTS);
    }
  }
  return MRV_OK;
}

// The work classes a batch may hold (bit c: class c, whose kernel instance
// is then launched).  Host batches are scanned (robots per query first;
// sphere sums only when the largest model could exceed a class bound);
// device batches may hold any.
static int batch_classes(const mrv_ctx *ctx, const mrv_batch *b) {
  if (b->flags & MRV_PTRS_ON_DEVICE) return (1 << kNumClasses) - 1;
  int n_max = 0;
  for (int q = 0; q < b->n_queries; ++q) n_max = std::max(n_max, b->q_robot_off[q + 1] - b->q_robot_off[q]);
  int m_max = 0;
  bool points = false;   // one-lane-per-state queries (point robots only) take the team class
  for (const auto &m : ctx->models) {
    m_max = std::max(m_max, m.dev.n_spheres);
    points |= m.dev.kind == MRV_ROBOT_POINT;
  }
  if (!points && work_class(n_max, n_max * m_max) == 0) return 1;
  const int n_models = (int)ctx->models.size();
  int mask = 0;
  for (int q = 0; q < b->n_queries; ++q) {
    int M = 0;
    bool all_point = true;
    const int n = b->q_robot_off[q + 1] - b->q_robot_off[q];
    for (int s = b->q_robot_off[q]; s < b->q_robot_off[q + 1]; ++s) {
      const int id = b->slot_robot_id[s];
      if (id >= 0 && id < n_models) {
        M += ctx->models[id].dev.n_spheres;
        all_point &= ctx->models[id].dev.kind == MRV_ROBOT_POINT;
      }
    }
    const int c = work_class(n, M);
    mask |= 1 << ((all_point && M <= kFlavorAMaxSpheres && c == 0) ? 1 : c);
  }
  return mask | 1;
}

BatchDev make_batchdev(mrv_ctx *ctx, const mrv_batch *b, Scratch &S, int forced_kind, int slices_per_item) {
  BatchDev B;
  std::memset(&B, 0, sizeof B);
  B.n_queries = b->n_queries;
  B.n_slots = b->n_slots;
  B.n_waypoints = b->n_waypoints;
  B.wp_stride = b->wp_stride;
  B.flags = b->flags;
  B.resolution = b->resolution;
  B.default_env = b->env_id == -1 ? -1 : ctx->env_slot(b->env_id);
  const bool dev = b->flags & MRV_PTRS_ON_DEVICE;
  B.q_robot_off = dev ? b->q_robot_off : S.in_q_off;
  B.slot_robot_id = dev ? b->slot_robot_id : S.in_slot_robot;
  B.slot_wp_off = dev ? b->slot_wp_off : S.in_slot_wp;
  B.waypoints = dev ? b->waypoints : S.in_wp;
  B.seg_steps = b->seg_steps ? (dev ? b->seg_steps : S.in_steps) : nullptr;
  B.q_env_id = b->q_env_id ? (dev ? b->q_env_id : S.in_q_env) : nullptr;
  B.q_kind = b->q_kind ? (dev ? b->q_kind : S.in_q_kind) : nullptr;
  B.forced_kind = forced_kind;
  B.slices_per_item = slices_per_item;
  B.tile_split = ctx->tuning.tile_split;
  B.mv_order = ctx->tuning.mv_order;
  B.slot_tau = S.slot_tau;
  B.q = S.q;
  B.q_hit = S.q_hit;
  B.q_best = S.q_best;
  B.q_minclr = S.q_minclr;
  B.sorted = S.sorted;
  B.redo_flag = S.redo_flag;
  B.redo = S.redo;
  B.q_states = S.q_states;
  B.hist = S.hist;
  B.level_start = S.level_start;
  B.cursor = S.cursor;
  B.counters = S.counters;
  B.err = S.err;
  B.stats = S.stats;
  B.models = ctx->d_models;
  B.n_models = (int32_t)ctx->models.size();
  B.envs = ctx->d_envs;
  B.n_envs = (int32_t)ctx->envs.size();
  B.clock_budget = ctx->clock_budget;
  B.classes = b->n_queries > 0 ? batch_classes(ctx, b) : 1;
  B.full = (b->flags & MRV_NO_BROADPHASE) ? 1 : 0;   // and every run asking for minimum clearances
  B.clr = 0;
  return B;
}

int stage_inputs(const mrv_batch *b, Scratch &S, cudaStream_t st) {
  if (b->flags & MRV_PTRS_ON_DEVICE) return MRV_OK;
  const int64_t nq = b->n_queries, ns = b->n_slots, nw = b->n_waypoints;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void *dst, const void *src, size_t n) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st);
  };
  cp(S.in_q_off, b->q_robot_off, sizeof(int32_t) * (nq + 1));
  cp(S.in_slot_robot, b->slot_robot_id, sizeof(int32_t) * ns);
  cp(S.in_slot_wp, b->slot_wp_off, sizeof(int32_t) * (ns + 1));
  cp(S.in_wp, b->waypoints, sizeof(float) * nw * b->wp_stride);
  if (b->seg_steps) cp(S.in_steps, b->seg_steps, sizeof(int32_t) * nw);
  if (b->q_env_id) cp(S.in_q_env, b->q_env_id, sizeof(int32_t) * nq);
  if (b->q_kind) cp(S.in_q_kind, b->q_kind, sizeof(uint8_t) * nq);
  if (e != cudaSuccess) return cuda_fail(e, "input copy");
  return MRV_OK;
}

cudaError_t Scratch::reset(cudaStream_t st) const {
  const char *a = reinterpret_cast<const char *>(hist);
  const char *b = reinterpret_cast<const char *>(counts + 4);
  const bool contiguous = a < reinterpret_cast<const char *>(level_start) &&
                          reinterpret_cast<const char *>(level_start) < reinterpret_cast<const char *>(cursor) &&
                          reinterpret_cast<const char *>(cursor) < reinterpret_cast<const char *>(counters) &&
                          reinterpret_cast<const char *>(counters) < reinterpret_cast<const char *>(err) &&
                          reinterpret_cast<const char *>(err) < reinterpret_cast<const char *>(stats) &&
                          reinterpret_cast<const char *>(stats) < reinterpret_cast<const char *>(counts) &&
                          b - a < (1 << 16);
  if (contiguous) return cudaMemsetAsync(hist, 0, (size_t)(b - a), st);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * kLevelBins, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(int32_t) * kNumCounters, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(uint32_t) * kErrWords, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * kNumStats, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * 4, st);
  return e;
}

int grid_for(mrv_ctx *ctx, int warps, bool full, int blocks_per_sm, int cls) {
  // the occupancy of a kernel configuration does not change: queried once
  int *slot = (warps >= 1 && warps <= 12 && cls >= 0 && cls < kNumClasses) ? &ctx->occ[full ? 1 : 0][cls][warps]
                                                                         : nullptr;
  int occ = slot ? *slot : 0;
  if (occ < 1) {
    if (max_blocks_per_sm(warps, full, cls, &occ) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    } else if (slot) {
      *slot = occ;
    }
  }
  if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
  return ctx->num_sms * occ;
}

// Issues the launch sequence on the context's stream (capturable).
// the full large-team instance over the queries the default instances
// handed over (usually none: its warps find the list empty and return)
cudaError_t launch_redo(mrv_ctx *ctx, const BatchDev &B, cudaStream_t st) {
  const int lw = large_warps();
  return launch_main(B, grid_for(ctx, lw, true, 1, 2), lw, true, 2, kRedoPass, st);
}

int enqueue_run(mrv_ctx *ctx, const BatchDev &B, Scratch &S, uint8_t *valid, float *minclr,
                mrv_conflict *conf, bool timed) {
  return enqueue_run_on(ctx, B, S, valid, minclr, conf, ctx->stream, timed ? ctx->ev0 : nullptr,
                        timed ? ctx->ev1 : nullptr, &ctx->fork);
}

int enqueue_run_on(mrv_ctx *ctx, const BatchDev &B, Scratch &S, uint8_t *valid, float *minclr,
                   mrv_conflict *conf, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, const Fork *fk) {
  const bool full = B.full != 0;   // the persistent kernel's full instances
  cudaGetLastError();   // the launch checks below report this sequence's errors only
  cudaError_t e = S.reset(st);
  if (e != cudaSuccess) return cuda_fail(e, "scratch reset");
  if ((e = launch_prepare(B, st)) != cudaSuccess) return cuda_fail(e, "prepare launch");
  const int warps = ctx->tuning.warps_per_block;
  if ((e = set_main_attrs(warps)) != cudaSuccess) return cuda_fail(e, "kernel attributes");
  // while the stream is captured, timing events must be external records to
  // become event nodes of the graph; outside capture they are plain records
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess) return cuda_fail(e, "capture status");
  const unsigned rec_flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ev0 && (e = cudaEventRecordWithFlags(ev0, st, rec_flags)) != cudaSuccess) return cuda_fail(e, "timing event");
  // the small-team instance on this stream; the team and large-team
  // instances, when the batch may hold their queries, on the fork's stream
  // beside it (after it on this stream without a fork)
  const int more = B.classes & ~1;
  const bool side = more && fk && fk->aux;
  if (side && (e = cudaEventRecord(fk->fork, st)) != cudaSuccess) return cuda_fail(e, "fork event");
  e = launch_main(B, grid_for(ctx, warps, full, ctx->tuning.blocks_per_sm, 0), warps, full, 0, -1, st);
  if (e != cudaSuccess) return cuda_fail(e, "main launch");
  if (more) {
    cudaStream_t ls = side ? fk->aux : st;
    if (side && (e = cudaStreamWaitEvent(ls, fk->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
    if (B.classes & 2) {
      e = launch_main(B, grid_for(ctx, warps, full, ctx->tuning.blocks_per_sm, 1), warps, full, 1, -1, ls);
      if (e != cudaSuccess) return cuda_fail(e, "team launch");
    }
    if (B.classes & 4) {
      const int lw = large_warps();
      e = launch_main(B, grid_for(ctx, lw, full, 0, 2), lw, full, 2, -1, ls);
      if (e != cudaSuccess) return cuda_fail(e, "large-team launch");
    }
    if (side && ((e = cudaEventRecord(fk->join, ls)) != cudaSuccess || (e = cudaStreamWaitEvent(st, fk->join, 0)) != cudaSuccess))
      return cuda_fail(e, "join");
  }
  if (!full && (e = launch_redo(ctx, B, st)) != cudaSuccess) return cuda_fail(e, "full-instance pass launch");
  if (ev1 && (e = cudaEventRecordWithFlags(ev1, st, rec_flags)) != cudaSuccess) return cuda_fail(e, "timing event");
  if ((e = launch_finish(B, valid, minclr, conf, S.counts, st)) != cudaSuccess) return cuda_fail(e, "finish launch");
  return MRV_OK;
}

static const char *check_site_name(uint32_t site) {
  static const char *const names[] = {"none",
#define MRV_CK_NAME(name, text) text,
                                      MRV_CHECK_SITES(MRV_CK_NAME)
#undef MRV_CK_NAME
  };
  return site < sizeof(names) / sizeof(names[0]) ? names[site] : "unknown site";
}

int check_device_err(const uint32_t *rec) {
  const uint32_t err = rec[0];
  if (!err) return MRV_OK;
  if (err & kErrChecked)
    return fail(MRV_ERR_CUDA, "bounds check failed (MRV_CHECKED build): %s, index %u outside 0..%u",
                check_site_name(rec[1]), rec[2], rec[3] ? rec[3] - 1 : 0u);
  if (err & kErrTimeout) return fail(MRV_ERR_TIMEOUT, "device work exceeded its clock budget");
  if (err & kErrAbort) return fail(MRV_ERR_TIMEOUT, "device work aborted");
  if (err & kErrRobotId) return fail(MRV_ERR_NOT_FOUND, "batch names an unknown robot id");
  if (err & kErrEnvId) return fail(MRV_ERR_NOT_FOUND, "batch names an unknown env id");
  if (err & kErrSpheres) return fail(MRV_ERR_LIMIT, "a query has more than %d spheres", MRV_MAX_QUERY_SPHERES);
  if (err & kErrSteps) return fail(MRV_ERR_LIMIT, "a query has bad step counts or T > %d", MRV_MAX_STEPS);
  if (err & kErrRobots) return fail(MRV_ERR_ARG, "a query has 0 or more than %d robots", MRV_MAX_ROBOTS);
  if (err & kErrWaypoints) return fail(MRV_ERR_ARG, "a slot has bad waypoint offsets or counts");
  if (err & kErrDof) return fail(MRV_ERR_ARG, "wp_stride is smaller than a robot's dof");
  return fail(MRV_ERR_ARG, "device reported error bits 0x%x", err);
}

int finish_call(mrv_ctx *ctx, Scratch &S, bool async) {
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(ctx->h_status, S.err, sizeof(uint32_t) * kErrWords, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_stats, S.stats, sizeof(unsigned long long) * kNumStats, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_counts, S.counts, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  ctx->pending = true;
  if (async) return MRV_OK;
  return ctx->sync();
}

}  // namespace mrv

using mrv::cuda_fail;

int mrv_ctx::sync() {
  using namespace mrv;
  cudaSetDevice(device);
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  if (!pending) return MRV_OK;
  pending = false;
  stats.sphere_tests = h_stats[1];
  stats.states_checked = h_stats[0];
  stats.states_available = h_stats[2];
  stats.sphere_tests_available = h_stats[3];
  stats.work_items = h_stats[4];
  stats.box_tests = h_stats[5];
  stats.fk_chains = h_stats[6];
  stats.spheres_placed = h_stats[7];
  stats.cylinder_tests = h_stats[8];
  stats.method_sphere_tests = h_stats[9];
  stats.method_box_tests = h_stats[10];
  stats.method_cylinder_tests = h_stats[11];
  stats.method_joints = h_stats[12];
  stats.method_chains = h_stats[13];
  stats.method_spheres = h_stats[14];
  stats.queries_redone = h_stats[15];
  stats.n_valid = h_counts[0];
  stats.n_conflicts = h_counts[1];
  float ms = 0.f;
  if (timed_pending && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) stats.device_ms = ms;
  cudaGetLastError();
  timed_pending = false;
  return check_device_err(h_status);
}

namespace mrv {

int run_batch(mrv_ctx *ctx, const mrv_batch *b, int forced_kind, uint8_t *valid, float *minclr,
              mrv_conflict *conf) {
  int rc = validate_batch(ctx, b);
  if (rc) return rc;
  if (b->n_queries == 0) {
    ctx->stats = mrv_stats{};
    return MRV_OK;
  }
  if (minclr && !(b->flags & MRV_EXHAUSTIVE))
    return fail(MRV_ERR_ARG, "min_clearance_out requires MRV_EXHAUSTIVE");
  if (ctx->pending && (rc = ctx->sync())) return rc;
  cudaSetDevice(ctx->device);
  Scratch &S = ctx->scratch;
  if ((rc = S.ensure(b->n_queries, b->n_slots, b->n_waypoints, b->wp_stride, ctx->stream))) return rc;
  if ((rc = stage_inputs(b, S, ctx->stream))) return rc;
  const bool dev = b->flags & MRV_PTRS_ON_DEVICE;
  const bool clr = minclr != nullptr;
  const bool per_query = b->flags & MRV_PER_QUERY_LAUNCH;
  BatchDev B = make_batchdev(ctx, b, S, forced_kind, per_query ? 1 : ctx->tuning.slices_per_item);
  if (clr) B.clr = B.full = 1;
  uint8_t *v_dst = valid ? (dev ? valid : S.out_valid) : nullptr;
  float *m_dst = minclr ? (dev ? minclr : S.out_minclr) : nullptr;
  mrv_conflict *c_dst = conf ? (dev ? conf : S.out_conf) : nullptr;
  cudaStream_t st = ctx->stream;
  if (!per_query) {
    if ((rc = enqueue_run(ctx, B, S, v_dst, m_dst, c_dst, true))) return rc;
  } else {
    // baseline: one synchronous launch per query (grid = the query's chunks)
    cudaError_t e = S.reset(st);
    if (e == cudaSuccess) e = launch_prepare(B, st);
    if (e != cudaSuccess) return cuda_fail(e, "prepare");
    std::vector<QueryDev> hq(b->n_queries);
    e = cudaMemcpyAsync(hq.data(), S.q, sizeof(QueryDev) * b->n_queries, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "query table copy");
    if ((e = set_main_attrs(1)) != cudaSuccess) return cuda_fail(e, "kernel attributes");
    cudaEventRecord(ctx->ev0, st);
    for (int q = 0; q < b->n_queries; ++q) {
      if (hq[q].bits & 4u || hq[q].nchunks == 0) continue;
      const int cls = (int)((hq[q].bits >> 3) & 3u);
      if ((e = launch_main(B, hq[q].nchunks, 1, B.full != 0, cls, q, st)) != cudaSuccess) return cuda_fail(e, "query launch");
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "query synchronize");
    }
    if (!B.full && (e = launch_redo(ctx, B, st)) != cudaSuccess) return cuda_fail(e, "full-instance pass launch");
    cudaEventRecord(ctx->ev1, st);
    if ((e = launch_finish(B, v_dst, m_dst, c_dst, S.counts, st)) != cudaSuccess) return cuda_fail(e, "finish");
  }
  ctx->timed_pending = true;
  if (!dev) {
    cudaError_t e = cudaSuccess;
    const size_t nq = b->n_queries;
    if (valid) e = cudaMemcpyAsync(valid, S.out_valid, nq, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && minclr) e = cudaMemcpyAsync(minclr, S.out_minclr, nq * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && conf) e = cudaMemcpyAsync(conf, S.out_conf, nq * sizeof(mrv_conflict), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
  }
  return finish_call(ctx, S, (b->flags & MRV_ASYNC) != 0);
}

// ---------------------------------------------------------------------------
// registry
// ---------------------------------------------------------------------------

}  // namespace mrv

int mrv_ctx::env_slot(int32_t id) const {
  using namespace mrv;
  const int s = id - kEnvIdBase;
  if (s < 0 || s >= (int)envs.size() || !envs[s].dev.live) return -1;
  return s;
}

int mrv_ctx::push_tables() {
  using namespace mrv;
  // every stream of the device may read the tables (contexts, servers)
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize before table update");
  auto grow = [&](void **dptr, size_t *cap, size_t need, size_t elem) -> cudaError_t {
    if (need <= *cap && *dptr) return cudaSuccess;
    size_t c = std::max<size_t>(16, need * 2);
    void *p = nullptr;
    cudaError_t r = dev_malloc(&p, c * elem);
    if (r != cudaSuccess) return r;
    if (*dptr) cudaFree(*dptr);
    *dptr = p;
    *cap = c;
    return cudaSuccess;
  };
  std::vector<ModelDev> hm(models.size());
  for (size_t i = 0; i < models.size(); ++i) hm[i] = models[i].dev;
  std::vector<EnvDev> he(envs.size());
  for (size_t i = 0; i < envs.size(); ++i) he[i] = envs[i].dev;
  if ((e = grow((void **)&d_models, &cap_models, hm.size(), sizeof(ModelDev))) != cudaSuccess)
    return cuda_fail(e, "model table");
  if ((e = grow((void **)&d_envs, &cap_envs, he.size(), sizeof(EnvDev))) != cudaSuccess) return cuda_fail(e, "env table");
  if (!hm.empty() && (e = cudaMemcpy(d_models, hm.data(), hm.size() * sizeof(ModelDev), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "model table copy");
  if (!he.empty() && (e = cudaMemcpy(d_envs, he.data(), he.size() * sizeof(EnvDev), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "env table copy");
  return MRV_OK;
}

namespace mrv {

static int upload(void **dst, const void *src, size_t n) {
  *dst = nullptr;
  if (n == 0) return MRV_OK;
  cudaError_t e = dev_malloc(dst, n);
  if (e != cudaSuccess) {
    *dst = nullptr;
    return cuda_fail(e, "upload allocation");
  }
  e = cudaMemcpy(*dst, src, n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "upload copy");
  return MRV_OK;
}

}  // namespace mrv

using namespace mrv;

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char *mrv_last_error(mrv_ctx *) { return g_err.c_str(); }

int mrv_create(mrv_ctx **out, int device, void *cuda_stream) {
  if (!out) return fail(MRV_ERR_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(MRV_ERR_CUDA, "no CUDA device available");
  }
  if (device < 0 || device >= n) return fail(MRV_ERR_ARG, "device %d outside 0..%d", device, n - 1);
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  mrv_ctx *c = new (std::nothrow) mrv_ctx();
  if (!c) return fail(MRV_ERR_OOM, "context allocation");
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) c->device_name = prop.name;
  e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e == cudaSuccess) e = c->fork.create();
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, 4096);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "context resources");
  }
  // pinned host words: status at 0, statistics at 64, counts at 256
  static_assert(64 + sizeof(unsigned long long) * kNumStats <= 256, "statistics fit before the counts");
  c->h_status = (uint32_t *)c->h_pinned;
  c->h_stats = (unsigned long long *)((char *)c->h_pinned + 64);
  c->h_counts = (int32_t *)((char *)c->h_pinned + 256);
  *out = c;
  return MRV_OK;
}

int mrv_destroy(mrv_ctx *c) {
  if (!c) return MRV_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto &m : c->models) m.free_all();
  for (auto &e : c->envs) e.free_all();
  c->scratch.release();
  if (c->d_models) cudaFree(c->d_models);
  if (c->d_envs) cudaFree(c->d_envs);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  c->fork.destroy();
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  delete c;
  return MRV_OK;
}

int mrv_set_stream(mrv_ctx *c, void *stream) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  int rc = c->sync();
  c->stream = (cudaStream_t)stream;
  return rc;
}

int robot_model_upload(mrv_ctx *c, const mrv_robot_desc *d, int32_t *id_out) {
  if (!c || !d || !id_out) return fail(MRV_ERR_ARG, "NULL argument");
  if (d->kind != MRV_ROBOT_DH_CHAIN && d->kind != MRV_ROBOT_POINT) return fail(MRV_ERR_ARG, "unknown robot kind");
  if (d->kind == MRV_ROBOT_DH_CHAIN && (d->dof < 1 || d->dof > MRV_MAX_DOF))
    return fail(MRV_ERR_LIMIT, "dof %d outside 1..%d", d->dof, MRV_MAX_DOF);
  if (d->kind == MRV_ROBOT_POINT && d->dof != 2 && d->dof != 3) return fail(MRV_ERR_ARG, "point robots have dof 2 or 3");
  if (d->kind == MRV_ROBOT_DH_CHAIN && !d->dh) return fail(MRV_ERR_ARG, "DH table missing");
  if (d->n_spheres < 1 || d->n_spheres > MRV_MAX_SPHERES)
    return fail(MRV_ERR_LIMIT, "n_spheres %d outside 1..%d", d->n_spheres, MRV_MAX_SPHERES);
  if (!d->sphere_link || !d->sphere_xyzr) return fail(MRV_ERR_ARG, "sphere arrays missing");
  if (d->n_self_pairs < 0 || (d->n_self_pairs > 0 && !d->self_pairs)) return fail(MRV_ERR_ARG, "self pairs missing");
  const int n_frames = d->kind == MRV_ROBOT_POINT ? 2 : d->dof + 2;
  for (int s = 0; s < d->n_spheres; ++s) {
    if (d->sphere_link[s] < 0 || d->sphere_link[s] >= n_frames)
      return fail(MRV_ERR_ARG, "sphere %d attached to frame %d (0..%d)", s, d->sphere_link[s], n_frames - 1);
    const float *x = d->sphere_xyzr + 4 * s;
    if (!(std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2]) && x[3] > 0.f && std::isfinite(x[3])))
      return fail(MRV_ERR_ARG, "sphere %d not finite or radius <= 0", s);
  }
  for (int p = 0; p < d->n_self_pairs; ++p) {
    const int a = d->self_pairs[2 * p], b = d->self_pairs[2 * p + 1];
    if (a < 0 || b < 0 || a >= d->n_spheres || b >= d->n_spheres || a == b)
      return fail(MRV_ERR_ARG, "self pair %d (%d, %d) invalid", p, a, b);
  }
  cudaSetDevice(c->device);
  HostModel m;
  ModelDev &D = m.dev;
  std::memset(&D, 0, sizeof D);
  D.kind = d->kind;
  D.dof = d->dof;
  D.n_spheres = d->n_spheres;
  D.n_self = d->n_self_pairs;
  D.live = 1;
  D.point_z = d->point_z;
  static const float I34[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  std::memcpy(D.base, d->base ? d->base : I34, sizeof D.base);
  std::memcpy(D.flange, d->flange ? d->flange : I34, sizeof D.flange);
  if (d->kind == MRV_ROBOT_DH_CHAIN)
    for (int k = 0; k < d->dof; ++k) {
      const float *r = d->dh + 4 * k;
      D.dh[k][0] = std::cos(r[1]);
      D.dh[k][1] = std::sin(r[1]);
      D.dh[k][2] = r[0];
      D.dh[k][3] = r[2];
      D.th0[k] = r[3];
    }
  for (int s = 0; s < d->n_spheres; ++s) D.r2max = std::max(D.r2max, d->sphere_xyzr[4 * s + 3] * d->sphere_xyzr[4 * s + 3]);
  // spheres grouped by frame with one bounding sphere per frame; self pairs
  // grouped by frame pair (the order within a group keeps neighbouring lanes
  // on the same or adjacent spheres)
  const int n_links = d->kind == MRV_ROBOT_POINT ? 2 : d->dof + 2;
  const PreparedModel PM = prepare_model(n_links, d->n_spheres, d->sphere_link, d->sphere_xyzr, d->n_self_pairs,
                                         d->self_pairs);
  const auto &sp = PM.self;
  // packed x | y << 16; the tail up to a multiple of 4 repeats the last pair
  // (a repeated pair changes no verdict)
  std::vector<uint32_t> spf((sp.size() + 3) / 4 * 4);
  for (size_t p = 0; p < spf.size(); ++p) {
    const auto &e = sp[std::min(p, sp.size() - 1)];
    spf[p] = (uint32_t)e.first | ((uint32_t)e.second << 16);
  }
  D.n_links = n_links;
  D.frame_mask = 0;
  for (int l = 0; l < n_links; ++l)
    if (PM.link_bs[4 * l + 3] >= 0.f) D.frame_mask |= 1u << l;
  for (int l = 0; l <= n_links; ++l) D.link_start[l] = PM.link_start[l];
  for (int l = 0; l < n_links; ++l)
    for (int k = 0; k < 4; ++k) D.link_bs[l][k] = PM.link_bs[4 * l + k];
  int rc;
  if ((rc = upload(&m.d_spheres, PM.spheres.data(), sizeof(float) * PM.spheres.size()))) return rc;
  if ((rc = upload(&m.d_links, PM.links.data(), sizeof(int32_t) * PM.links.size()))) { m.free_all(); return rc; }
  if ((rc = upload(&m.d_self, spf.data(), sizeof(uint32_t) * spf.size()))) { m.free_all(); return rc; }
  if ((rc = upload(&m.d_groups, PM.self_groups.data(), sizeof(int32_t) * PM.self_groups.size()))) {
    m.free_all();
    return rc;
  }
  if ((rc = upload(&m.d_perm, PM.perm.data(), sizeof(int32_t) * PM.perm.size()))) { m.free_all(); return rc; }
  if ((rc = upload(&m.d_blocks, PM.self_blocks.data(), sizeof(int32_t) * PM.self_blocks.size())) ||
      (rc = upload(&m.d_masks, PM.self_masks.data(), sizeof(uint32_t) * PM.self_masks.size()))) {
    m.free_all();
    return rc;
  }
  D.self_blocks = PM.self_blocks.empty() ? nullptr : (const int4 *)m.d_blocks;
  D.self_masks = PM.self_masks.empty() ? nullptr : (const uint32_t *)m.d_masks;
  D.n_masks = (int32_t)PM.self_masks.size();
  // rectangles pay off only when they are large enough to fill a warp's
  // 4-rows-per-lane tiling; small ones stay on the sparse pair path
  std::vector<std::pair<int32_t, int32_t>> spr(sp);
  std::sort(spr.begin(), spr.end());
  std::vector<int32_t> rects = self_pair_rectangles(d->n_spheres, spr, 256);
  if (!rects.empty() && (int64_t)sp.size() < 64 * (int64_t)(rects.size() / 4)) rects.clear();
  if ((rc = upload(&m.d_rects, rects.data(), sizeof(int32_t) * rects.size()))) { m.free_all(); return rc; }
  D.self_rects = (const int4 *)m.d_rects;
  D.n_rects = (int32_t)rects.size() / 4;
  D.self_groups = (const int4 *)m.d_groups;
  D.n_groups = (int32_t)PM.self_groups.size() / 4;
  D.perm = (const int32_t *)m.d_perm;
  D.spheres = (const float4 *)m.d_spheres;
  D.sphere_link = (const int32_t *)m.d_links;
  D.self_pairs = (const uint32_t *)m.d_self;
  m.refs = 1;
  m.max_spheres = d->n_spheres;
  c->models.push_back(m);
  if ((rc = c->push_tables())) {
    c->models.back().free_all();
    c->models.pop_back();
    return rc;
  }
  *id_out = (int32_t)c->models.size() - 1;
  return MRV_OK;
}

int env_upload(mrv_ctx *c, const mrv_env_desc *d, int32_t *id_out) {
  if (!c || !d || !id_out) return fail(MRV_ERR_ARG, "NULL argument");
  if (d->n_spheres < 0 || d->n_aabbs < 0 || d->n_cylinders < 0) return fail(MRV_ERR_ARG, "negative obstacle counts");
  if ((d->n_spheres && !d->spheres_xyzr) || (d->n_aabbs && !d->aabb_lohi) || (d->n_cylinders && !d->cylinders))
    return fail(MRV_ERR_ARG, "obstacle arrays missing");
  // cylinders: finite, radius >= 0, distinct axis ends; stored as (a, radius)
  // and (unit axis, length), computed in double
  std::vector<float> cyl_a(4 * (size_t)d->n_cylinders), cyl_u(4 * (size_t)d->n_cylinders);
  for (int i = 0; i < d->n_cylinders; ++i) {
    const float *x = d->cylinders + 7 * i;
    for (int k = 0; k < 7; ++k)
      if (!std::isfinite(x[k])) return fail(MRV_ERR_ARG, "cylinder %d not finite", i);
    if (!(x[6] >= 0.f)) return fail(MRV_ERR_ARG, "cylinder %d has a negative radius", i);
    double u[3], L = 0.0;
    for (int k = 0; k < 3; ++k) {
      u[k] = (double)x[3 + k] - (double)x[k];
      L += u[k] * u[k];
    }
    L = std::sqrt(L);
    if (!(L > 0.0)) return fail(MRV_ERR_ARG, "cylinder %d has coinciding axis ends", i);
    for (int k = 0; k < 3; ++k) {
      cyl_a[4 * i + k] = x[k];
      cyl_u[4 * i + k] = (float)(u[k] / L);
    }
    cyl_a[4 * i + 3] = x[6];
    cyl_u[4 * i + 3] = (float)L;
  }
  for (int i = 0; i < d->n_aabbs; ++i)
    for (int k = 0; k < 3; ++k)
      if (!(d->aabb_lohi[6 * i + k] <= d->aabb_lohi[6 * i + 3 + k]))
        return fail(MRV_ERR_ARG, "box %d has lo > hi on axis %d", i, k);
  cudaSetDevice(c->device);
  for (int i = 0; i < d->n_spheres; ++i) {
    const float *x = d->spheres_xyzr + 4 * i;
    if (!(std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2]) && std::isfinite(x[3]) && x[3] >= 0.f))
      return fail(MRV_ERR_ARG, "obstacle sphere %d not finite or radius < 0", i);
  }
  HostEnv h;
  std::memset(&h.dev, 0, sizeof h.dev);
  // per obstacle sphere k = |c|^2 - r^2 (double, rounded once), and the
  // largest |c|^2 and r^2 that bound the rounding of the kernel's test
  std::vector<float> k(d->n_spheres);
  double c2max = 0.0, r2max = 0.0;
  for (int i = 0; i < d->n_spheres; ++i) {
    const float *x = d->spheres_xyzr + 4 * i;
    const double c2 = (double)x[0] * x[0] + (double)x[1] * x[1] + (double)x[2] * x[2];
    const double r2 = (double)x[3] * x[3];
    k[i] = (float)(c2 - r2);
    c2max = std::max(c2max, c2);
    r2max = std::max(r2max, r2);
  }
  std::vector<float> lo(4 * (size_t)d->n_aabbs), hi(4 * (size_t)d->n_aabbs);
  for (int i = 0; i < d->n_aabbs; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[4 * i + a] = d->aabb_lohi[6 * i + a];
      hi[4 * i + a] = d->aabb_lohi[6 * i + 3 + a];
    }
  int rc;
  if ((rc = upload(&h.d_spheres, d->spheres_xyzr, sizeof(float) * 4 * d->n_spheres))) return rc;
  if ((rc = upload(&h.d_k, k.data(), sizeof(float) * k.size()))) { h.free_all(); return rc; }
  if ((rc = upload(&h.d_lo, lo.data(), sizeof(float) * lo.size()))) { h.free_all(); return rc; }
  if ((rc = upload(&h.d_hi, hi.data(), sizeof(float) * hi.size()))) { h.free_all(); return rc; }
  h.dev.n_spheres = d->n_spheres;
  h.dev.n_aabbs = d->n_aabbs;
  h.dev.live = 1;
  h.dev.c2max = (float)(c2max * (1.0 + 1e-6));
  h.dev.r2max = (float)(r2max * (1.0 + 1e-6));
  h.dev.spheres = (const float4 *)h.d_spheres;
  h.dev.sphere_k = (const float *)h.d_k;
  h.dev.box_lo = (const float4 *)h.d_lo;
  h.dev.box_hi = (const float4 *)h.d_hi;
  // obstacle grid for frames up to the largest frame bounding radius of the
  // robot models uploaded so far (0.3 m without any); larger frames of
  // models uploaded later scan every obstacle
  float R = 0.f;
  for (const HostModel &m : c->models)
    if (m.dev.live)
      for (int l = 0; l < m.dev.n_links; ++l) R = std::max(R, m.dev.link_bs[l][3]);
  if (!(R > 0.f)) R = 0.3f;
  const ObstacleGrid G = build_obstacle_grid(d->n_spheres, d->spheres_xyzr, d->n_aabbs, d->aabb_lohi,
                                             d->n_cylinders, d->cylinders, (double)R);
  if ((rc = upload(&h.d_cyla, cyl_a.data(), sizeof(float) * cyl_a.size())) ||
      (rc = upload(&h.d_cylu, cyl_u.data(), sizeof(float) * cyl_u.size()))) {
    h.free_all();
    return rc;
  }
  h.dev.n_cyl = d->n_cylinders;
  h.dev.cyl_a = (const float4 *)h.d_cyla;
  h.dev.cyl_u = (const float4 *)h.d_cylu;
  h.dev.g_R = -1.f;
  if (G.R > 0) {
    std::vector<uint32_t> cnt(G.ns.size());
    for (size_t c = 0; c < cnt.size(); ++c) cnt[c] = (uint32_t)G.ns[c] | ((uint32_t)G.nb[c] << 16);
    if ((rc = upload(&h.d_goff, G.off.data(), sizeof(int32_t) * G.off.size())) ||
        (rc = upload(&h.d_gcnt, cnt.data(), sizeof(uint32_t) * cnt.size())) ||
        (rc = upload(&h.d_gitems, G.items.data(), sizeof(uint16_t) * std::max<size_t>(1, G.items.size())))) {
      h.free_all();
      return rc;
    }
    for (int a = 0; a < 3; ++a) {
      h.dev.g_lo[a] = (float)G.lo[a];
      h.dev.g_dims[a] = G.dims[a];
    }
    h.dev.g_inv_h = (float)(1.0 / G.h);
    h.dev.g_R = R;
    h.dev.g_off = (const int32_t *)h.d_goff;
    h.dev.g_cnt = (const uint32_t *)h.d_gcnt;
    h.dev.g_items = (const uint16_t *)h.d_gitems;
    h.dev.g_nitems = (int32_t)G.items.size();
  }
  h.refs = 1;
  c->envs.push_back(h);
  if ((rc = c->push_tables())) {
    c->envs.back().free_all();
    c->envs.pop_back();
    return rc;
  }
  *id_out = kEnvIdBase + (int32_t)c->envs.size() - 1;
  return MRV_OK;
}

int mrv_release(mrv_ctx *c, int32_t id) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  cudaSetDevice(c->device);
  if (id >= kEnvIdBase) {
    const int s = c->env_slot(id);
    if (s < 0) return fail(MRV_ERR_NOT_FOUND, "unknown env id %d", id);
    if (--c->envs[s].refs == 0) {
      int rc = c->sync();
      c->envs[s].free_all();
      c->envs[s].dev.live = 0;
      int rc2 = c->push_tables();
      return rc ? rc : rc2;
    }
    return MRV_OK;
  }
  if (id < 0 || id >= (int)c->models.size() || !c->models[id].dev.live)
    return fail(MRV_ERR_NOT_FOUND, "unknown robot id %d", id);
  if (--c->models[id].refs == 0) {
    int rc = c->sync();
    c->models[id].free_all();
    c->models[id].dev.live = 0;
    int rc2 = c->push_tables();
    return rc ? rc : rc2;
  }
  return MRV_OK;
}

int mv_validate(mrv_ctx *c, const mrv_batch *b, uint8_t *valid_out, float *min_clearance_out) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  if (!valid_out && b && b->n_queries > 0) return fail(MRV_ERR_ARG, "valid_out is NULL");
  return run_batch(c, b, MRV_KIND_MV, valid_out, min_clearance_out, nullptr);
}

int ffc_find(mrv_ctx *c, const mrv_batch *b, mrv_conflict *out) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  if (!out && b && b->n_queries > 0) return fail(MRV_ERR_ARG, "out is NULL");
  return run_batch(c, b, MRV_KIND_FFC, nullptr, nullptr, out);
}

int mrv_run(mrv_ctx *c, const mrv_batch *b, uint8_t *valid_out, mrv_conflict *conflict_out) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  if (b && b->n_queries > 0 && (!valid_out || !conflict_out)) return fail(MRV_ERR_ARG, "outputs are NULL");
  if (b && b->n_queries > 0 && !b->q_kind) return fail(MRV_ERR_ARG, "mrv_run needs q_kind");
  return run_batch(c, b, -1, valid_out, nullptr, conflict_out);
}

int mrv_sync(mrv_ctx *c) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  return c->sync();
}

int mrv_set_limits(mrv_ctx *c, const mrv_limits *l) {
  if (!c || !l) return fail(MRV_ERR_ARG, "NULL argument");
  if (!(l->kernel_budget_ms >= 0.0) || l->kernel_budget_ms > 1e9) return fail(MRV_ERR_ARG, "budget outside 0..1e9 ms");
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device) != cudaSuccess || khz <= 0) {
    cudaGetLastError();
    khz = 2070000;   // the GB300's maximum SM clock, a safe upper bound on ticks per ms
  }
  c->clock_budget = l->kernel_budget_ms > 0.0 ? (long long)(l->kernel_budget_ms * khz) : 0;
  if (l->kernel_budget_ms > 0.0 && c->clock_budget < 1) c->clock_budget = 1;
  return MRV_OK;
}

int mrv_get_stats(mrv_ctx *c, mrv_stats *out) {
  if (!c || !out) return fail(MRV_ERR_ARG, "NULL argument");
  *out = c->stats;
  return MRV_OK;
}

int mrv_set_tuning(mrv_ctx *c, const mrv_tuning *t) {
  if (!c || !t) return fail(MRV_ERR_ARG, "NULL argument");
  if (t->slices_per_item < 1 || t->slices_per_item > 4096) return fail(MRV_ERR_ARG, "slices_per_item outside 1..4096");
  if (t->warps_per_block < 1 || t->warps_per_block > 12) return fail(MRV_ERR_ARG, "warps_per_block outside 1..12");
  if (t->blocks_per_sm < 0) return fail(MRV_ERR_ARG, "blocks_per_sm < 0");
  if (t->tile_split < 1 || t->tile_split > 32 || (t->tile_split & (t->tile_split - 1)))
    return fail(MRV_ERR_ARG, "tile_split must be 1, 2, 4, 8, 16 or 32");
  if (t->mv_order < 0 || t->mv_order > 1) return fail(MRV_ERR_ARG, "mv_order must be 0 or 1");
  c->tuning = *t;
  return MRV_OK;
}

int mrv_get_tuning(mrv_ctx *c, mrv_tuning *t) {
  if (!c || !t) return fail(MRV_ERR_ARG, "NULL argument");
  *t = c->tuning;
  return MRV_OK;
}

int mrv_clearance(mrv_ctx *c, const mrv_batch *b, int32_t q, const int32_t *ts, int32_t nt, float *out) {
  if (!c) return fail(MRV_ERR_ARG, "ctx is NULL");
  int rc = validate_batch(c, b);
  if (rc) return rc;
  if (q < 0 || q >= b->n_queries) return fail(MRV_ERR_ARG, "query %d outside the batch", q);
  if (nt < 0 || (nt > 0 && (!ts || !out))) return fail(MRV_ERR_ARG, "bad timestep list");
  if (nt == 0) return MRV_OK;
  if (c->pending && (rc = c->sync())) return rc;
  cudaSetDevice(c->device);
  Scratch &S = c->scratch;
  if ((rc = S.ensure(b->n_queries, b->n_slots, b->n_waypoints, b->wp_stride, c->stream))) return rc;
  if ((rc = stage_inputs(b, S, c->stream))) return rc;
  const bool dev = b->flags & MRV_PTRS_ON_DEVICE;
  BatchDev B = make_batchdev(c, b, S, MRV_KIND_MV, 1);
  cudaStream_t st = c->stream;
  cudaError_t e = S.reset(st);
  if (e == cudaSuccess) e = launch_prepare(B, st);
  if (e != cudaSuccess) return cuda_fail(e, "prepare");
  // the query's sphere count bounds the output; read it back
  QueryDev hq;
  if ((e = cudaMemcpyAsync(&hq, S.q + q, sizeof hq, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "query record copy");
  if (hq.bits & 4u) {
    uint32_t rec[kErrWords] = {};
    cudaMemcpy(rec, S.err, sizeof rec, cudaMemcpyDeviceToHost);
    if (!rec[0]) rec[0] = kErrRobots;
    return check_device_err(rec);
  }
  const int32_t *d_ts = ts;
  float *d_out = out;
  void *tmp = nullptr;
  if (!dev) {
    const size_t bytes = sizeof(int32_t) * nt + sizeof(float) * (size_t)nt * hq.M;
    if ((e = dev_malloc(&tmp, bytes)) != cudaSuccess) return cuda_fail(e, "clearance buffers");
    d_ts = (const int32_t *)tmp;
    d_out = (float *)((char *)tmp + sizeof(int32_t) * nt);
    e = cudaMemcpyAsync((void *)d_ts, ts, sizeof(int32_t) * nt, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = launch_clearance(B, q, d_ts, nt, (b->flags & MRV_CHECK_ENV) ? 1 : 0, d_out, st);
  if (e == cudaSuccess && !dev)
    e = cudaMemcpyAsync(out, d_out, sizeof(float) * (size_t)nt * hq.M, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_status, S.err, sizeof(uint32_t) * kErrWords, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "clearance");
  return check_device_err(c->h_status);
}

// ---- graphs -----------------------------------------------------------------

int mrv_graph_create(mrv_ctx *c, const mrv_batch *b, uint8_t *valid_out, mrv_conflict *conflict_out,
                     mrv_graph **out) {
  if (!c || !out) return fail(MRV_ERR_ARG, "NULL argument");
  *out = nullptr;
  int rc = validate_batch(c, b);
  if (rc) return rc;
  if (!(b->flags & MRV_PTRS_ON_DEVICE)) return fail(MRV_ERR_ARG, "graphs need MRV_PTRS_ON_DEVICE");
  if (b->flags & MRV_PER_QUERY_LAUNCH) return fail(MRV_ERR_ARG, "graphs replay the batched path only");
  if (b->n_queries == 0) return fail(MRV_ERR_ARG, "empty batch");
  if (!b->q_kind || !valid_out || !conflict_out) return fail(MRV_ERR_ARG, "graphs capture mrv_run: q_kind and both outputs needed");
  if (c->pending && (rc = c->sync())) return rc;
  cudaSetDevice(c->device);
  mrv_graph *g = new (std::nothrow) mrv_graph();
  if (!g) return fail(MRV_ERR_OOM, "graph allocation");
  g->ctx = c;
  if ((rc = g->scratch.ensure(b->n_queries, b->n_slots, b->n_waypoints, b->wp_stride, c->stream))) {
    delete g;
    return rc;
  }
  BatchDev B = make_batchdev(c, b, g->scratch, -1, c->tuning.slices_per_item);
  // attributes are set outside the capture
  set_main_attrs(c->tuning.warps_per_block);
  grid_for(c, c->tuning.warps_per_block, B.full != 0, c->tuning.blocks_per_sm, 0);
  grid_for(c, c->tuning.warps_per_block, B.full != 0, c->tuning.blocks_per_sm, 1);
  grid_for(c, large_warps(), B.full != 0, 0, 2);
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g->scratch.release();
    delete g;
    return cuda_fail(e, "capture stream");
  }
  cudaStream_t saved = c->stream;
  c->stream = cap;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = enqueue_run(c, B, g->scratch, valid_out, nullptr, conflict_out, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (rc == MRV_OK && e2 == cudaSuccess) {
      e2 = cudaGraphInstantiate(&g->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e2 != cudaSuccess) rc = cuda_fail(e2, "graph instantiate");
    } else if (rc == MRV_OK) {
      rc = cuda_fail(e2, "graph capture");
    }
  } else {
    rc = cuda_fail(e, "begin capture");
  }
  c->stream = saved;
  cudaStreamDestroy(cap);
  if (rc) {
    g->scratch.release();
    delete g;
    return rc;
  }
  *out = g;
  return MRV_OK;
}

int mrv_graph_launch(mrv_graph *g) {
  if (!g || !g->exec) return fail(MRV_ERR_ARG, "graph is NULL");
  mrv_ctx *c = g->ctx;
  cudaSetDevice(c->device);
  cudaError_t e = cudaGraphLaunch(g->exec, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  // status of the replay is read by the next mrv_sync
  e = cudaMemcpyAsync(c->h_status, g->scratch.err, sizeof(uint32_t) * kErrWords, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_stats, g->scratch.stats, sizeof(unsigned long long) * kNumStats, cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_counts, g->scratch.counts, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph status copy");
  c->pending = true;
  c->timed_pending = true;   // the graph records the context's timing events
  return MRV_OK;
}

int mrv_graph_destroy(mrv_graph *g) {
  if (!g) return MRV_OK;
  cudaSetDevice(g->ctx->device);
  cudaStreamSynchronize(g->ctx->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->scratch.release();
  delete g;
  return MRV_OK;
}

}  // extern "C"
