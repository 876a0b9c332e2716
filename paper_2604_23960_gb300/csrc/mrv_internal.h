// Host-side types of the runtime (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mrv_dev.h"
#include "mrv_geometry.h"

namespace mrv {

extern thread_local std::string g_err;
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
cudaError_t dev_malloc(void **p, size_t n);   // cudaMalloc with test fault injection

// device scratch of one run: derived per-query arrays, counters, staged
// inputs and outputs; one arena, grown on demand, carved at 256-byte offsets
struct Scratch {
  void *base = nullptr;
  size_t cap = 0;
  int32_t *slot_tau = nullptr;
  QueryDev *q = nullptr;
  int32_t *q_hit = nullptr, *q_best = nullptr;
  float *q_minclr = nullptr;
  int32_t *sorted = nullptr, *hist = nullptr, *level_start = nullptr, *cursor = nullptr;
  int32_t *redo_flag = nullptr, *redo = nullptr, *q_states = nullptr;
  int32_t *counters = nullptr;
  uint32_t *err = nullptr;
  unsigned long long *stats = nullptr;
  int32_t *counts = nullptr;
  int32_t *in_q_off = nullptr, *in_slot_robot = nullptr, *in_slot_wp = nullptr, *in_steps = nullptr,
          *in_q_env = nullptr;
  float *in_wp = nullptr;
  uint8_t *in_q_kind = nullptr;
  uint8_t *out_valid = nullptr;
  float *out_minclr = nullptr;
  mrv_conflict *out_conf = nullptr;

  static size_t bytes_for(int64_t nq, int64_t ns, int64_t nw, int64_t stride);
  // the arena's layout: sets every pointer from p (nothing when p is null)
  // and returns the bytes spanned; bytes_for and ensure both use it
  size_t layout(int64_t nq, int64_t ns, int64_t nw, int64_t stride, char *p);
  int ensure(int64_t nq, int64_t ns, int64_t nw, int64_t stride, cudaStream_t st);
  void release();
  // zeroes the per-call state (level bins, counters, error word, statistics,
  // result counts), which every carving lays out back to back: one memset
  cudaError_t reset(cudaStream_t st) const;
};

struct HostModel {
  ModelDev dev{};
  void *d_spheres = nullptr, *d_links = nullptr, *d_self = nullptr, *d_rects = nullptr, *d_groups = nullptr,
       *d_perm = nullptr, *d_blocks = nullptr, *d_masks = nullptr;
  int refs = 0;
  int max_spheres = 0;
  void free_all() {
    for (void **p : {&d_spheres, &d_links, &d_self, &d_rects, &d_groups, &d_perm, &d_blocks, &d_masks}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
  }
};



struct HostEnv {
  EnvDev dev{};
  void *d_spheres = nullptr, *d_k = nullptr, *d_lo = nullptr, *d_hi = nullptr;
  void *d_goff = nullptr, *d_gcnt = nullptr, *d_gitems = nullptr;   // obstacle grid
  void *d_cyla = nullptr, *d_cylu = nullptr;                                          // cylinders
  int refs = 0;
  void free_all() {
    for (void **p : {&d_spheres, &d_k, &d_lo, &d_hi, &d_goff, &d_gcnt, &d_gitems, &d_cyla, &d_cylu}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
  }
};

// A second stream beside a work stream for the large-team kernel instance:
// it runs concurrently with the team instance (its one-per-SM blocks start as
// the team kernel's blocks leave their SMs, and return at once when the batch
// holds no such query) and is joined back before the result kernel.
struct Fork {
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    return e;
  }
  void destroy() {
    if (aux) cudaStreamSynchronize(aux);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (aux) cudaStreamDestroy(aux);
    aux = nullptr;
    fork = join = nullptr;
  }
};

// kernel launch wrappers (mrv_kernels.cu)
size_t main_smem_bytes(int warps, int cls);   // cls: work class (0 small team, 1 team, 2 large team)
int large_warps();                             // warps per block of the large-team instance
cudaError_t launch_prepare(const BatchDev &B, cudaStream_t st);
cudaError_t set_main_attrs(int warps);
cudaError_t max_blocks_per_sm(int warps, bool full, int cls, int *out);
cudaError_t launch_main(const BatchDev &B, int grid, int warps, bool full, int cls, int q_single, cudaStream_t st);
cudaError_t launch_finish(const BatchDev &B, uint8_t *valid, float *minclr, mrv_conflict *conf, int *counts,
                          cudaStream_t st);
cudaError_t launch_clearance(const BatchDev &B, int q, const int32_t *ts, int nt, int check_env, float *out,
                             cudaStream_t st);

}  // namespace mrv

struct mrv_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  std::string device_name;
  std::vector<mrv::HostModel> models;
  std::vector<mrv::HostEnv> envs;
  mrv::ModelDev *d_models = nullptr;
  mrv::EnvDev *d_envs = nullptr;
  size_t cap_models = 0, cap_envs = 0;
  mrv::Scratch scratch;
  mrv_tuning tuning{1, 4, 0, 4, 0};
  mrv_stats stats{};
  long long clock_budget = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  mrv::Fork fork;               // second stream of the large-team instance
  int occ[2][mrv::kNumClasses][13] = {};   // resident blocks per SM by [full instance][class][warps] (0: not queried yet)
  void *h_pinned = nullptr;
  uint32_t *h_status = nullptr;
  unsigned long long *h_stats = nullptr;
  int32_t *h_counts = nullptr;
  bool pending = false, timed_pending = false;

  int env_slot(int32_t id) const;
  int push_tables();
  int sync();
};

struct mrv_graph {
  mrv_ctx *ctx = nullptr;
  cudaGraphExec_t exec = nullptr;
  mrv::Scratch scratch;
};

namespace mrv {
int validate_batch(mrv_ctx *ctx, const mrv_batch *b);
BatchDev make_batchdev(mrv_ctx *ctx, const mrv_batch *b, Scratch &S, int forced_kind, int slices_per_item);
int enqueue_run(mrv_ctx *ctx, const BatchDev &B, Scratch &S, uint8_t *valid, float *minclr,
                mrv_conflict *conf, bool timed);
int enqueue_run_on(mrv_ctx *ctx, const BatchDev &B, Scratch &S, uint8_t *valid, float *minclr,
                   mrv_conflict *conf, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, const Fork *fk);
int stage_inputs(const mrv_batch *b, Scratch &S, cudaStream_t st);
int run_batch(mrv_ctx *ctx, const mrv_batch *b, int forced_kind, uint8_t *valid, float *minclr, mrv_conflict *conf);
int grid_for(mrv_ctx *ctx, int warps, bool full, int blocks_per_sm, int cls);
// maps a device error record (kErrWords words) to a status and message
int check_device_err(const uint32_t *rec);
// copies the error word, statistics and counts of the call just enqueued to
// the context's pinned host words; waits for them unless async
int finish_call(mrv_ctx *ctx, Scratch &S, bool async);
}  // namespace mrv
