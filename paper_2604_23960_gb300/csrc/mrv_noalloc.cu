// MotionValidation without any allocation during the call.
//
// Some callers cannot allocate device memory when they validate motions: a
// planner running inside a latency-bounded control loop (cudaMalloc and
// cudaFree can block and cudaFree synchronizes the whole device), or a host
// application whose device memory is owned by another allocator and fully
// budgeted.  This entry point runs the same preparation, persistent and
// result kernels as mv_validate, but every piece of per-call scratch lives in
// one file-scope device array reserved when the library's device code is
// loaded, so the call itself allocates nothing.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; each call re-initialises all of it that must start from a
// known value (counters, error word, histograms by memset; per-query records
// and waypoint times are rewritten by the preparation kernel).  Two calls
// whose work overlaps on the same device race on the array: issue them on one
// stream, or synchronize between them.
#include <cuda_runtime.h>

#include <cstring>

#include "mrv_internal.h"

namespace mrv {
namespace {

// per-call scratch: waypoint times, per-query records and verdict words,
// the sorted query list, the handed-over query list and its flags, level
// tables, counters, error word and statistics
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
constexpr size_t kBytes =
    align_up(sizeof(int32_t) * MRV_NOALLOC_MAX_WAYPOINTS) + align_up(sizeof(QueryDev) * MRV_NOALLOC_MAX_QUERIES) +
    6 * align_up(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES) + align_up(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES) +
    2 * align_up(sizeof(int32_t) * kLevelBins) + align_up(sizeof(int32_t) * 2 * kLevelBins) + align_up(sizeof(int32_t) * kNumCounters) + align_up(sizeof(uint32_t) * kErrWords) +
    align_up(sizeof(unsigned long long) * kNumStats) + align_up(sizeof(int32_t) * 4);

static __device__ __align__(256) unsigned char g_scratch[kBytes];

// The address of g_scratch on the current device (host code cannot use the
// symbol itself as a device pointer).  Looked up on every call: the lookup
// allocates nothing, and a cached address would go stale if the device's
// primary context were ever recreated (cudaDeviceReset).
int scratch_address(void **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "scratch symbol address");
  *out = p;
  return MRV_OK;
}

// Points a Scratch view at the static array (no staging buffers: inputs and
// outputs are the caller's device arrays).
void carve(void *base, int64_t nq, int64_t nw, Scratch *S) {
  char *p = static_cast<char *>(base);
  size_t o = 0;
  auto take = [&](size_t n) {
    void *r = p + o;
    o += align_up(n);
    return r;
  };
  S->slot_tau = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_WAYPOINTS);
  S->q = (QueryDev *)take(sizeof(QueryDev) * MRV_NOALLOC_MAX_QUERIES);
  S->q_hit = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES);
  S->q_best = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES);
  S->q_minclr = (float *)take(sizeof(float) * MRV_NOALLOC_MAX_QUERIES);
  S->sorted = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES);
  S->redo_flag = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES);
  S->redo = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES);
  S->q_states = (int32_t *)take(sizeof(int32_t) * MRV_NOALLOC_MAX_QUERIES);
  S->hist = (int32_t *)take(sizeof(int32_t) * kLevelBins);
  S->level_start = (int32_t *)take(sizeof(int32_t) * kLevelBins);
  S->cursor = (int32_t *)take(sizeof(int32_t) * 2 * kLevelBins);
  S->counters = (int32_t *)take(sizeof(int32_t) * kNumCounters);
  S->err = (uint32_t *)take(sizeof(uint32_t) * kErrWords);
  S->stats = (unsigned long long *)take(sizeof(unsigned long long) * kNumStats);
  S->counts = (int32_t *)take(sizeof(int32_t) * 4);
  (void)nq;
  (void)nw;
}

}  // namespace
}  // namespace mrv

using namespace mrv;

extern "C" int mv_validate_noalloc(mrv_ctx *ctx, const mrv_batch *b, uint8_t *valid_out) {
  if (!ctx || !b) return fail(MRV_ERR_ARG, "NULL argument");
  if (!(b->flags & MRV_PTRS_ON_DEVICE))
    return fail(MRV_ERR_ARG, "mv_validate_noalloc takes device pointers only (set MRV_PTRS_ON_DEVICE)");
  if (b->flags & (MRV_ASYNC | MRV_PER_QUERY_LAUNCH | MRV_EXHAUSTIVE))
    return fail(MRV_ERR_ARG, "mv_validate_noalloc runs the synchronous batched early-exit path only");
  int rc = validate_batch(ctx, b);
  if (rc) return rc;
  if (b->n_queries == 0) return MRV_OK;
  if (!valid_out) return fail(MRV_ERR_ARG, "valid_out is NULL");
  if (b->n_queries > MRV_NOALLOC_MAX_QUERIES)
    return fail(MRV_ERR_LIMIT, "%d queries exceed the allocation-free maximum of %d", b->n_queries,
                MRV_NOALLOC_MAX_QUERIES);
  if (b->n_waypoints > MRV_NOALLOC_MAX_WAYPOINTS)
    return fail(MRV_ERR_LIMIT, "%d waypoints exceed the allocation-free maximum of %d", b->n_waypoints,
                MRV_NOALLOC_MAX_WAYPOINTS);
  if (ctx->pending && (rc = ctx->sync())) return rc;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  // the call waits for its result, which a stream under capture cannot do
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(ctx->stream, &cs)) != cudaSuccess) return cuda_fail(e, "capture status");
  if (cs != cudaStreamCaptureStatusNone)
    return fail(MRV_ERR_ARG, "mv_validate_noalloc cannot run on a stream that is being captured");
  void *base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  Scratch S;   // a view only: it owns nothing (base stays null)
  carve(base, b->n_queries, b->n_waypoints, &S);
  const BatchDev B = make_batchdev(ctx, b, S, MRV_KIND_MV, ctx->tuning.slices_per_item);
  if ((rc = enqueue_run_on(ctx, B, S, valid_out, nullptr, nullptr, ctx->stream, ctx->ev0, ctx->ev1,
                           &ctx->fork)))
    return rc;
  // error word, statistics and counts come back through the context's pinned
  // host words, as for every other call (mrv_get_stats then describes this one)
  ctx->timed_pending = true;
  return finish_call(ctx, S, false);
}
