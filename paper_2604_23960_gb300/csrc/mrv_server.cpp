// Serving loop: continuous batching of MV / FFC requests over CUDA streams.
//
// Clients submit host batches (copied at submission).  A scheduler thread
// admits waiting requests in arrival order whenever a stream slot is free and
// the request's device footprint fits in the unused part of the budget;
// compatible requests (same batch form, resolution and flags) are packed into
// one micro-batch, staged through the slot's pinned buffer and run with the
// same preparation + persistent kernels as mrv_run.  Micro-batches on
// different slots overlap on the device; completions are detected with
// events, results are split back per request and waiting clients woken.
// Every wait is bounded (condition variables with timeouts, event polling);
// nothing spins on the device.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "mrv_internal.h"

namespace mrv {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int32_t nq = 0, ns = 0, nw = 0, stride = 0;
  std::vector<int32_t> q_off, slot_robot, slot_wp, steps, q_env;
  std::vector<float> wp;
  std::vector<uint8_t> kind;
  bool timed = false, has_env = false, has_kind = false;
  float resolution = 0.f;
  uint32_t flags = 0;
  int32_t env_id = -1;
  size_t footprint = 0;
  std::vector<uint8_t> valid;
  std::vector<mrv_conflict> conf;
  int status = MRV_OK;
  std::string message;
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  Scratch scratch;
  void *pin_in = nullptr;
  size_t pin_in_cap = 0;
  void *pin_out = nullptr;
  size_t pin_out_cap = 0;
  cudaEvent_t done_ev = nullptr, ev0 = nullptr, ev1 = nullptr;
  Fork fork;   // second stream of the large-team instance
  std::vector<std::shared_ptr<Request>> reqs;
  int32_t nq = 0;
  size_t footprint = 0;
  bool busy = false;
  int launch_status = MRV_OK;
  std::string launch_msg;
};

static bool compatible(const Request &a, const Request &b) {
  return a.timed == b.timed && a.flags == b.flags && (a.timed || a.resolution == b.resolution);
}

static int grow_pinned(void **p, size_t *cap, size_t need) {
  if (need <= *cap) return MRV_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  size_t want = need + need / 2 + 4096;
  cudaError_t e = cudaMallocHost(p, want);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "pinned staging");
  }
  *cap = want;
  return MRV_OK;
}

// pinned staging of one micro-batch: packed inputs, and results (valid
// bytes rounded up to 256, conflicts, the error word)
static size_t in_bytes_for(size_t nq, size_t ns, size_t nw, size_t stride, bool timed) {
  return sizeof(int32_t) * (nq + 1 + ns + ns + 1 + (timed ? nw : 0) + nq) + sizeof(float) * nw * stride + nq +
         64 * 8;
}
static size_t out_bytes_for(size_t nq) { return ((nq + 255) & ~size_t(255)) + sizeof(mrv_conflict) * nq + 64; }
static_assert(sizeof(uint32_t) * kErrWords <= 64, "the error record fits the result staging's tail");

}  // namespace mrv

struct mrv_server {
  mrv_ctx *ctx = nullptr;
  mrv_server_opts opts{};
  std::vector<mrv::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<mrv::Request>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<mrv::Request>> table;
  size_t used = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  mrv_server_stats st{};
  uint64_t inflight = 0;

  void loop();
  void launch(mrv::Slot &s);
  void complete(mrv::Slot &s);
};

using namespace mrv;

// Packs the slot's requests into one micro-batch in pinned memory and issues
// copies, kernels and result copies on the slot's stream.
void mrv_server::launch(Slot &s) {
  cudaGetLastError();   // a launch reports its own errors only
  int32_t nq = 0, ns = 0, nw = 0, stride = 1;
  bool timed = s.reqs[0]->timed, any_env = false, any_kind = false;
  for (auto &r : s.reqs) {
    nq += r->nq;
    ns += r->ns;
    nw += r->nw;
    stride = std::max(stride, r->stride);
    any_env |= r->has_env || r->env_id != -1;
    any_kind |= r->has_kind;
  }
  const size_t in_bytes = in_bytes_for(nq, ns, nw, stride, timed);
  const size_t out_bytes = out_bytes_for(nq);
  // buffers were sized at creation; they grow here only for a single request
  // larger than that (the packing below never exceeds them otherwise)
  int rc = grow_pinned(&s.pin_in, &s.pin_in_cap, in_bytes);
  if (!rc) rc = grow_pinned(&s.pin_out, &s.pin_out_cap, out_bytes);
  if (!rc) rc = s.scratch.ensure(nq, ns, nw, stride, s.stream);
  if (rc) {
    s.launch_status = rc;
    s.launch_msg = g_err;
    cudaEventRecord(s.done_ev, s.stream);
    return;
  }
  char *p = (char *)s.pin_in;
  auto carve = [&](size_t n) {
    char *r = p;
    p += (n + 63) & ~size_t(63);
    return r;
  };
  int32_t *q_off = (int32_t *)carve(sizeof(int32_t) * (nq + 1));
  int32_t *slot_robot = (int32_t *)carve(sizeof(int32_t) * ns);
  int32_t *slot_wp = (int32_t *)carve(sizeof(int32_t) * (ns + 1));
  int32_t *steps = timed ? (int32_t *)carve(sizeof(int32_t) * nw) : nullptr;
  int32_t *q_env = (int32_t *)carve(sizeof(int32_t) * nq);
  float *wp = (float *)carve(sizeof(float) * (size_t)nw * stride);
  uint8_t *kind = (uint8_t *)carve(nq);
  int32_t qb = 0, sb = 0, wb = 0;
  q_off[0] = 0;
  slot_wp[0] = 0;
  for (auto &r : s.reqs) {
    for (int q = 0; q < r->nq; ++q) {
      q_off[qb + q + 1] = sb + r->q_off[q + 1];
      q_env[qb + q] = r->has_env ? r->q_env[q] : r->env_id;
      kind[qb + q] = r->has_kind ? r->kind[q] : (uint8_t)MRV_KIND_MV;
    }
    for (int k = 0; k < r->ns; ++k) {
      slot_robot[sb + k] = r->slot_robot[k];
      slot_wp[sb + k + 1] = wb + r->slot_wp[k + 1];
    }
    for (int w = 0; w < r->nw; ++w) {
      std::memcpy(wp + (size_t)(wb + w) * stride, r->wp.data() + (size_t)w * r->stride, sizeof(float) * r->stride);
      for (int k = r->stride; k < stride; ++k) wp[(size_t)(wb + w) * stride + k] = 0.f;
      if (timed) steps[wb + w] = r->steps[w];
    }
    qb += r->nq;
    sb += r->ns;
    wb += r->nw;
  }
  (void)any_kind;
  mrv_batch b{};
  b.n_queries = nq;
  b.n_slots = ns;
  b.n_waypoints = nw;
  b.env_id = -1;
  b.q_robot_off = q_off;
  b.slot_robot_id = slot_robot;
  b.slot_wp_off = slot_wp;
  b.waypoints = wp;
  b.wp_stride = stride;
  b.seg_steps = steps;
  b.resolution = s.reqs[0]->resolution;
  b.q_env_id = any_env ? q_env : nullptr;
  b.q_kind = kind;
  b.flags = s.reqs[0]->flags & (MRV_CHECK_ENV | MRV_EXHAUSTIVE);
  s.nq = nq;
  rc = stage_inputs(&b, s.scratch, s.stream);
  uint8_t *valid_h = (uint8_t *)s.pin_out;
  mrv_conflict *conf_h = (mrv_conflict *)((char *)s.pin_out + (((size_t)nq + 255) & ~size_t(255)));
  uint32_t *err_h = (uint32_t *)((char *)conf_h + sizeof(mrv_conflict) * (size_t)nq);
  if (!rc) {
    BatchDev B = make_batchdev(ctx, &b, s.scratch, -1, ctx->tuning.slices_per_item);
    rc = enqueue_run_on(ctx, B, s.scratch, s.scratch.out_valid, nullptr, s.scratch.out_conf, s.stream, s.ev0,
                        s.ev1, &s.fork);
  }
  if (!rc) {
    int which = 0;
    cudaError_t e = cudaMemcpyAsync(valid_h, s.scratch.out_valid, nq, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) {
      which = 1;
      e = cudaMemcpyAsync(conf_h, s.scratch.out_conf, sizeof(mrv_conflict) * nq, cudaMemcpyDeviceToHost, s.stream);
    }
    if (e == cudaSuccess) {
      which = 2;
      e = cudaMemcpyAsync(err_h, s.scratch.err, sizeof(uint32_t) * kErrWords, cudaMemcpyDeviceToHost, s.stream);
    }
    if (e != cudaSuccess) {
      // what the runtime knows about the buffers, for the error report
      auto kind = [](const void *p) {
        cudaPointerAttributes a{};
        const cudaError_t pe = cudaPointerGetAttributes(&a, p);
        cudaGetLastError();
        return pe == cudaSuccess ? (int)a.type : -1 - (int)pe;
      };
      const cudaError_t sq = cudaStreamQuery(s.stream);
      cudaGetLastError();
      char what[320];
      std::snprintf(what, sizeof what,
                    "server result copy %d (%d queries; host %p cap %zu type %d, conf %d..%d; device %p %p %p types "
                    "%d %d %d; stream %d)",
                    which, nq, s.pin_out, s.pin_out_cap, kind(s.pin_out), kind(conf_h),
                    kind((char *)conf_h + sizeof(mrv_conflict) * nq - 1), (void *)s.scratch.out_valid,
                    (void *)s.scratch.out_conf, (void *)s.scratch.err, kind(s.scratch.out_valid),
                    kind(s.scratch.out_conf), kind(s.scratch.err), (int)sq);
      rc = cuda_fail(e, what);
    }
  }
  if (rc) {
    s.launch_status = rc;
    s.launch_msg = g_err;
  }
  cudaEventRecord(s.done_ev, s.stream);
}

// Splits a finished micro-batch's results back to its requests.
void mrv_server::complete(Slot &s) {
  int rc = s.launch_status;
  std::string msg = s.launch_msg;
  const int32_t nq = s.nq;
  uint8_t *valid_h = (uint8_t *)s.pin_out;
  mrv_conflict *conf_h = (mrv_conflict *)((char *)s.pin_out + (((size_t)nq + 255) & ~size_t(255)));
  uint32_t *err_h = (uint32_t *)((char *)conf_h + sizeof(mrv_conflict) * (size_t)nq);
  if (!rc) {
    cudaError_t e = cudaEventQuery(s.done_ev);
    if (e != cudaSuccess) rc = cuda_fail(e, "micro-batch");
    else if (*err_h) rc = check_device_err(err_h);
    if (rc) msg = g_err;
  }
  float ms = 0.f;
  if (!rc && cudaEventElapsedTime(&ms, s.ev0, s.ev1) == cudaSuccess) st.busy_ms += ms;
  cudaGetLastError();
  int32_t qb = 0;
  for (auto &r : s.reqs) {
    r->status = rc;
    r->message = msg;
    if (!rc) {
      r->valid.assign(valid_h + qb, valid_h + qb + r->nq);
      r->conf.assign(conf_h + qb, conf_h + qb + r->nq);
    }
    qb += r->nq;
    r->done = true;
    used -= r->footprint;
    ++st.completed;
  }
  s.reqs.clear();
  s.busy = false;
  s.launch_status = MRV_OK;
  s.launch_msg.clear();
  --inflight;
}

void mrv_server::loop() {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool progressed = false;
    for (auto &s : slots)
      if (s.busy && cudaEventQuery(s.done_ev) != cudaErrorNotReady) {
        complete(s);
        progressed = true;
      }
    if (progressed) cv_done.notify_all();
    if (stop && pending.empty() && inflight == 0) break;
    for (auto &s : slots) {
      if (s.busy || pending.empty()) continue;
      // admission in arrival order: the head request decides the group
      auto &head = pending.front();
      if (used + head->footprint > opts.device_budget_bytes) break;
      int32_t q = 0, ns = 0, nw = 0, stride = 1;
      while (!pending.empty()) {
        auto &r = pending.front();
        if (!s.reqs.empty() && !compatible(*s.reqs[0], *r)) break;
        if (!s.reqs.empty() && q + r->nq > opts.max_batch_queries) break;
        if (used + r->footprint > opts.device_budget_bytes) break;
        // keep a micro-batch inside the slot's buffers (sized at creation),
        // so nothing is allocated while other micro-batches are in flight
        const int32_t st2 = std::max(stride, r->stride);
        if (!s.reqs.empty() &&
            (Scratch::bytes_for(q + r->nq, ns + r->ns, nw + r->nw, st2) > s.scratch.cap ||
             in_bytes_for(q + r->nq, ns + r->ns, nw + r->nw, st2, r->timed) > s.pin_in_cap ||
             out_bytes_for(q + r->nq) > s.pin_out_cap))
          break;
        ns += r->ns;
        nw += r->nw;
        stride = st2;
        used += r->footprint;
        q += r->nq;
        s.reqs.push_back(r);
        pending.pop_front();
      }
      s.busy = true;
      ++inflight;
      ++st.micro_batches;
      st.queries += q;
      if (inflight > st.max_inflight) st.max_inflight = inflight;
      lk.unlock();
      launch(s);
      lk.lock();
      progressed = true;
    }
    if (!progressed) cv_work.wait_for(lk, std::chrono::microseconds(inflight ? 50 : 2000));
  }
}

extern "C" {

int mrv_server_create(mrv_ctx *c, const mrv_server_opts *o, mrv_server **out) {
  if (!c || !o || !out) return fail(MRV_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (o->n_streams < 1 || o->n_streams > 16) return fail(MRV_ERR_ARG, "n_streams outside 1..16");
  if (o->max_batch_queries < 1 || o->max_pending < 1) return fail(MRV_ERR_ARG, "limits must be positive");
  if (o->device_budget_bytes == 0) return fail(MRV_ERR_ARG, "device budget is 0");
  cudaSetDevice(c->device);
  auto *s = new (std::nothrow) mrv_server();
  if (!s) return fail(MRV_ERR_OOM, "server allocation");
  s->ctx = c;
  s->opts = *o;
  s->slots.resize(o->n_streams);
  for (auto &sl : s->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.ev1);
    if (e == cudaSuccess) e = sl.fork.create();
    if (e != cudaSuccess) {
      int rc = cuda_fail(e, "server streams");
      mrv_server_destroy(s);
      return rc;
    }
  }
  // Every slot's device arena and pinned staging are sized here for a full
  // micro-batch of max_batch_queries queries of up to kTeamRobots robots on
  // two waypoints each (stride 8), within half of the free device memory, so
  // the scheduler allocates nothing while micro-batches are in flight (a
  // cudaFree or cudaFreeHost there would synchronize the whole device).
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "device memory query");
    mrv_server_destroy(s);
    return rc;
  }
  int64_t nq0 = o->max_batch_queries;
  auto arena = [](int64_t nq) { return Scratch::bytes_for(nq, nq * kTeamRobots, 2 * nq * kTeamRobots, 8); };
  while (nq0 > 256 && (size_t)o->n_streams * (arena(nq0) + arena(nq0) / 4) > free_b / 2) nq0 /= 2;
  for (auto &sl : s->slots) {
    int rc = sl.scratch.ensure(nq0, nq0 * kTeamRobots, 2 * nq0 * kTeamRobots, 8, sl.stream);
    if (!rc) rc = grow_pinned(&sl.pin_in, &sl.pin_in_cap, in_bytes_for(nq0, nq0 * kTeamRobots, 2 * nq0 * kTeamRobots, 8, true));
    if (!rc) rc = grow_pinned(&sl.pin_out, &sl.pin_out_cap, out_bytes_for(nq0));
    if (rc) {
      mrv_server_destroy(s);
      return rc;
    }
  }
  // admission by device memory: the budget cannot exceed what the device
  // holds for requests (its free memory now plus the arenas just sized)
  size_t free_after = 0;
  if ((e = cudaMemGetInfo(&free_after, &total_b)) != cudaSuccess) {
    int rc = cuda_fail(e, "device memory query");
    mrv_server_destroy(s);
    return rc;
  }
  size_t arenas = 0;
  for (auto &sl : s->slots) arenas += sl.scratch.cap;
  s->opts.device_budget_bytes = std::min(o->device_budget_bytes, free_after + arenas);
  s->st.device_budget_bytes = s->opts.device_budget_bytes;
  s->st.device_free_bytes = free_after;
  s->st.presized_queries = (uint64_t)nq0;
  try {
    s->th = std::thread([s] { s->loop(); });
  } catch (...) {
    mrv_server_destroy(s);
    return fail(MRV_ERR_OOM, "scheduler thread");
  }
  *out = s;
  return MRV_OK;
}

int mrv_server_destroy(mrv_server *s) {
  if (!s) return MRV_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->ctx->device);
  for (auto &sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    sl.scratch.release();
    if (sl.pin_in) cudaFreeHost(sl.pin_in);
    if (sl.pin_out) cudaFreeHost(sl.pin_out);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.ev0) cudaEventDestroy(sl.ev0);
    if (sl.ev1) cudaEventDestroy(sl.ev1);
    sl.fork.destroy();
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
  return MRV_OK;
}

int mrv_server_submit(mrv_server *s, const mrv_batch *b, uint64_t *ticket) {
  if (!s || !b || !ticket) return fail(MRV_ERR_ARG, "NULL argument");
  if (b->flags & ~(uint32_t)(MRV_CHECK_ENV | MRV_EXHAUSTIVE))
    return fail(MRV_ERR_ARG, "server requests take host batches with MRV_CHECK_ENV / MRV_EXHAUSTIVE only");
  int rc = validate_batch(s->ctx, b);
  if (rc) return rc;
  if (b->n_queries == 0) return fail(MRV_ERR_ARG, "empty request");
  auto r = std::make_shared<Request>();
  r->nq = b->n_queries;
  r->ns = b->n_slots;
  r->nw = b->n_waypoints;
  r->stride = b->wp_stride;
  r->q_off.assign(b->q_robot_off, b->q_robot_off + r->nq + 1);
  r->slot_robot.assign(b->slot_robot_id, b->slot_robot_id + r->ns);
  r->slot_wp.assign(b->slot_wp_off, b->slot_wp_off + r->ns + 1);
  r->wp.assign(b->waypoints, b->waypoints + (size_t)r->nw * r->stride);
  r->timed = b->seg_steps != nullptr;
  if (r->timed) r->steps.assign(b->seg_steps, b->seg_steps + r->nw);
  r->has_env = b->q_env_id != nullptr;
  if (r->has_env) r->q_env.assign(b->q_env_id, b->q_env_id + r->nq);
  r->has_kind = b->q_kind != nullptr;
  if (r->has_kind) r->kind.assign(b->q_kind, b->q_kind + r->nq);
  r->resolution = b->resolution;
  r->flags = b->flags;
  r->env_id = b->env_id;
  r->footprint = Scratch::bytes_for(r->nq, r->ns, r->nw, r->stride);
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->footprint > s->opts.device_budget_bytes) {
    ++s->st.rejected;
    return fail(MRV_ERR_BUSY, "request footprint %zu exceeds the device budget %zu", r->footprint,
                s->opts.device_budget_bytes);
  }
  if ((int)s->pending.size() >= s->opts.max_pending) {
    ++s->st.rejected;
    return fail(MRV_ERR_BUSY, "%d requests already waiting", (int)s->pending.size());
  }
  if (s->stop) return fail(MRV_ERR_BUSY, "server is stopping");
  r->ticket = s->next_ticket++;
  s->table[r->ticket] = r;
  s->pending.push_back(r);
  ++s->st.submitted;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return MRV_OK;
}

int mrv_server_wait(mrv_server *s, uint64_t ticket, int32_t timeout_ms, uint8_t *valid_out,
                    mrv_conflict *conflict_out) {
  if (!s) return fail(MRV_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return fail(MRV_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (!r->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
      return fail(MRV_ERR_TIMEOUT, "request %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
  }
  s->table.erase(ticket);
  if (r->status) return fail(r->status, "%s", r->message.c_str());
  if (valid_out) std::memcpy(valid_out, r->valid.data(), r->valid.size());
  if (conflict_out) std::memcpy(conflict_out, r->conf.data(), sizeof(mrv_conflict) * r->conf.size());
  return MRV_OK;
}

int mrv_server_get_stats(mrv_server *s, mrv_server_stats *out) {
  if (!s || !out) return fail(MRV_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return MRV_OK;
}

}  // extern "C"
