// Kernels of multi-robot MotionValidation (MV, Alg. 1) and FindFirstConflict
// (FFC, Alg. 2) for sm_103a.
//
// Work decomposition
//   tile   32 states of one query, the GPU's batch of W = 32 timesteps
//          (PackCfgBatch, Sec. III-A): MV packs them with the rake order
//          t = b + nb*l (nb = ceil((T+1)/32)), FFC with the linear order
//          t = 32b + l.
//   chunk  consecutive tiles of one query, processed in order by one warp,
//          stopping as soon as the query is decided (MV: any collision;
//          FFC: a conflict in an earlier state).
//   item   one chunk; items are handed out by a global atomic counter in
//          level order: every query's first chunk, then every query's second
//          chunk, ... (queries sorted by chunk count), so coarse rake tiles
//          and early FFC timesteps of all queries run first.
// Two per-query flavors:
//   A  (point robots, <= 16 spheres): lane l owns state t(l) of the tile and
//      runs every check of that state; a ballot finds the first conflicting
//      lane.
//   B  (kinematic chains): the warp walks the tile's states; per FK round
//      16 lanes run the (state, robot) chains into shared-memory link frames,
//      then per state the lanes place the spheres and split the sphere-pair
//      rows; __any_sync / __reduce_or_sync reduce the verdict.
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "mrv_dev.h"

namespace mrv {

constexpr int kFlavorAMaxSpheres = 16;
constexpr int kSlotWords = 16;  // ints per RobotSlot in shared memory

struct RobotSlot {           // per-warp staged view of one robot of the query
  const float4 *spheres;
  const int32_t *links;
  const int2 *self;
  int32_t mdl, m, dof, kind, n_self, w0, w1, pad;
};
static_assert(sizeof(RobotSlot) <= kSlotWords * 4, "slot size");

struct WarpSmem {
  RobotSlot rs[MRV_MAX_ROBOTS];
  int32_t off[MRV_MAX_ROBOTS + 1];
  int32_t pad[7];
  // union region: flavor B frames + positions, or flavor A per-lane spheres
  union {
    struct {
      float xf[kFkChains * kMaxLinks * 12];
      float4 P[MRV_MAX_QUERY_SPHERES];
    } b;
    float4 PA[kFlavorAMaxSpheres * kWarp];
  } u;
};

__host__ __device__ constexpr size_t warp_smem_bytes() { return (sizeof(WarpSmem) + 15) & ~size_t(15); }

__device__ __forceinline__ int pair_index(int i, int j, int n) { return i * n - i * (i + 1) / 2 + (j - i - 1); }

// ordered-int encoding of floats so that atomicMin on int orders like floats
__device__ __forceinline__ int f2ord(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

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

__global__ void k_prep(BatchDev B) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B.n_queries) return;
  uint32_t err = 0;
  QueryDev Q;
  Q.T = 0; Q.n = 0; Q.M = 0; Q.ntiles = 0; Q.nchunks = 0; Q.cte = 1; Q.env = -1; Q.bits = 0;
  Q.pairtests = 0; Q.envtests = 0;
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
  long long self_total = 0;
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
      if (m.kind != MRV_ROBOT_POINT) all_point = false;
      const int w0 = B.slot_wp_off[s], w1 = B.slot_wp_off[s + 1];
      if (w0 < 0 || w1 <= w0 || w1 > B.n_waypoints) { err |= kErrWaypoints; break; }
      long long Ts = 0;
      if (B.seg_steps) {
        B.slot_tau[w0] = 0;
        for (int w = w0; w < w1 - 1; ++w) {
          const int st = B.seg_steps[w];
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
    if (all_point && M <= kFlavorAMaxSpheres) Q.bits |= 2u;
    Q.ntiles = (int)((T + 1 + kWarp - 1) / kWarp);
    int cte = B.chunk_tiles < 1 ? 1 : B.chunk_tiles;
    const int need = (Q.ntiles + kMaxLevels - 1) / kMaxLevels;
    if (cte < need) cte = need;
    Q.cte = cte;
    Q.nchunks = (Q.ntiles + cte - 1) / cte;
    long long pt = 0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) pt += (long long)ms[i] * ms[j];
    Q.pairtests = pt;
    long long et = 0;
    const bool mv = !(Q.bits & 1u);
    if (mv && (B.flags & MRV_CHECK_ENV)) {
      if (env >= 0) et = (long long)M * (B.envs[env].n_spheres + B.envs[env].n_aabbs);
      et += self_total;
    }
    Q.envtests = et;
    atomicAdd(&B.stats[2], (unsigned long long)(T + 1));
    atomicAdd(&B.stats[3], (unsigned long long)((T + 1) * (pt + et)));
  }
  B.q[q] = Q;
  B.q_hit[q] = 0;
  B.q_best[q] = 0x7fffffff;
  B.q_minclr[q] = __int_as_float(f2ord(INFINITY));
  atomicAdd(&B.hist[Q.nchunks > kMaxLevels ? kMaxLevels : Q.nchunks], 1);
}

// level layout: queries sorted by chunk count (descending); level c holds the
// queries with more than c chunks, which are the first cnt_c sorted queries.
__global__ void k_levels(BatchDev B) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int start = 0;
  for (int k = kMaxLevels; k >= 0; --k) {
    B.cursor[k] = start;           // first sorted position of chunk count k
    start += B.hist[k];
  }
  int acc = 0;
  B.level_start[0] = 0;
  for (int c = 0; c < kMaxLevels; ++c) {
    acc += B.cursor[c];            // queries with more than c chunks
    B.level_start[c + 1] = acc;
  }
  B.counters[1] = acc;             // number of work items
}

__global__ void k_scatter(BatchDev B) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B.n_queries) return;
  int c = B.q[q].nchunks;
  if (c > kMaxLevels) c = kMaxLevels;
  const int pos = atomicAdd(&B.cursor[c], 1);
  B.sorted[pos] = q;
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
    const float *a = B.waypoints + (size_t)last * B.wp_stride;
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
__device__ void chain_frames(const ModelDev &m, const float *q, float *X) {
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
      const float ca = m.dh[k][0], sa = m.dh[k][1], a = m.dh[k][2], d = m.dh[k][3], th0 = m.dh[k][4];
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

__device__ __forceinline__ bool sph_hit(const float4 a, const float4 b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float rr = a.w + b.w;
  return dx * dx + dy * dy + dz * dz < rr * rr;
}

__device__ __forceinline__ float sph_clr(const float4 a, const float4 b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return sqrtf(dx * dx + dy * dy + dz * dz) - (a.w + b.w);
}

__device__ __forceinline__ float box_d2(const float4 a, const float *bx) {
  const float ex = fmaxf(fmaxf(bx[0] - a.x, a.x - bx[3]), 0.f);
  const float ey = fmaxf(fmaxf(bx[1] - a.y, a.y - bx[4]), 0.f);
  const float ez = fmaxf(fmaxf(bx[2] - a.z, a.z - bx[5]), 0.f);
  return ex * ex + ey * ey + ez * ez;
}

// ---------------------------------------------------------------------------
// tile processing
// ---------------------------------------------------------------------------

struct TileCtx {
  int q, T, n, M, nb, ffc, check_env, exhaustive;
  int env_ns, env_nb;
  const float4 *env_s;
  const float *env_b;
  long long pairtests, envtests;
  unsigned long long tests, states;
};

__device__ __forceinline__ int tile_state(const TileCtx &C, int b, int l) {
  return C.ffc ? b * kWarp + l : b + C.nb * l;
}

// result of a tile: MV -> 1 if a collision was found; FFC -> key or INT_MAX
template <bool CLR>
__device__ int tile_flavor_a(const BatchDev &B, TileCtx &C, WarpSmem &S, int b, int lane, float &minclr) {
  const int t = tile_state(C, b, lane);
  const bool valid = t <= C.T;
  float4 *PA = S.u.PA;
  if (valid) {
    for (int r = 0; r < C.n; ++r) {
      const RobotSlot &rs = S.rs[r];
      const ModelDev &m = B.models[rs.mdl];
      float q[MRV_MAX_DOF];
      interp(B, rs.w0, rs.w1, rs.dof, t, q);
      const float z = rs.dof == 2 ? m.point_z : q[2];
      for (int k = 0; k < rs.m; ++k) {
        const float4 s = rs.spheres[k];
        float lx = s.x, ly = s.y, lz = s.z;
        if (rs.links[k] == 1) { lx += q[0]; ly += q[1]; lz += z; }
        float4 w;
        w.x = m.base[0] * lx + m.base[1] * ly + m.base[2] * lz + m.base[3];
        w.y = m.base[4] * lx + m.base[5] * ly + m.base[6] * lz + m.base[7];
        w.z = m.base[8] * lx + m.base[9] * ly + m.base[10] * lz + m.base[11];
        w.w = s.w;
        PA[(S.off[r] + k) * kWarp + lane] = w;
      }
    }
  }
  const int nvalid = __popc(__ballot_sync(0xffffffffu, valid));
  C.states += nvalid;
  if (!C.ffc) {
    bool hit = false;
    if (valid && C.check_env) {
      for (int a = 0; a < C.M; ++a) {
        const float4 pa = PA[a * kWarp + lane];
        for (int o = 0; o < C.env_ns; ++o) {
          if (CLR) minclr = fminf(minclr, sph_clr(pa, C.env_s[o]));
          else hit |= sph_hit(pa, C.env_s[o]);
        }
        for (int o = 0; o < C.env_nb; ++o) {
          const float d2 = box_d2(pa, C.env_b + 6 * o);
          if (CLR) minclr = fminf(minclr, sqrtf(d2) - pa.w);
          else hit |= d2 < pa.w * pa.w;
        }
      }
      for (int r = 0; r < C.n; ++r)
        for (int p = 0; p < S.rs[r].n_self; ++p) {
          const int2 sp = S.rs[r].self[p];
          const float4 x = PA[(S.off[r] + sp.x) * kWarp + lane], y = PA[(S.off[r] + sp.y) * kWarp + lane];
          if (CLR) minclr = fminf(minclr, sph_clr(x, y));
          else hit |= sph_hit(x, y);
        }
    }
    if (valid)
      for (int i = 0; i < C.n; ++i)
        for (int a = S.off[i]; a < S.off[i + 1]; ++a) {
          const float4 pa = PA[a * kWarp + lane];
          for (int bb = S.off[i + 1]; bb < C.M; ++bb) {
            const float4 pb = PA[bb * kWarp + lane];
            if (CLR) minclr = fminf(minclr, sph_clr(pa, pb));
            else hit |= sph_hit(pa, pb);
          }
        }
    C.tests += (unsigned long long)nvalid * (unsigned long long)(C.pairtests + (C.check_env ? C.envtests : 0));
    if (CLR) hit = minclr < 0.f;
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
  C.tests += (unsigned long long)nvalid * (unsigned long long)C.pairtests;
  const unsigned m = __ballot_sync(0xffffffffu, first != 0x7fffffff);
  if (!m) return 0x7fffffff;
  const int l0 = __ffs(m) - 1;
  const int p0 = __shfl_sync(0xffffffffu, first, l0);
  return tile_state(C, b, l0) * 32 + p0;
}

template <bool CLR>
__device__ int tile_flavor_b(const BatchDev &B, TileCtx &C, WarpSmem &S, int b, int lane, float &minclr) {
  const int n = C.n, M = C.M;
  const int CS = (kFkChains / n) < 1 ? 1 : (kFkChains / n);   // states per FK round
  float *xf = S.u.b.xf;
  float4 *P = S.u.b.P;
  const int rows = S.off[n - 1];
  int found = C.ffc ? 0x7fffffff : 0;
  for (int l0 = 0; l0 < kWarp; l0 += CS) {
    if (tile_state(C, b, l0) > C.T) break;   // states grow with l in both orders
    // (state, robot) chains
    if (lane < CS * n) {
      const int l = l0 + lane / n, r = lane % n;
      const int t = tile_state(C, b, l);
      if (l < kWarp && t <= C.T) {
        const RobotSlot &rs = S.rs[r];
        float q[MRV_MAX_DOF];
        interp(B, rs.w0, rs.w1, rs.dof, t, q);
        chain_frames(B.models[rs.mdl], q, xf + lane * (kMaxLinks * 12));
      }
    }
    __syncwarp();
    for (int l = l0; l < l0 + CS && l < kWarp; ++l) {
      const int t = tile_state(C, b, l);
      if (t > C.T) break;
      C.states += 1;
      // sphere placement
      for (int a = lane; a < M; a += kWarp) {
        int r = 0;
        while (a >= S.off[r + 1]) ++r;
        const int k = a - S.off[r];
        const float4 s = S.rs[r].spheres[k];
        const float *X = xf + ((l - l0) * n + r) * (kMaxLinks * 12) + S.rs[r].links[k] * 12;
        float4 w;
        w.x = fmaf(X[0], s.x, fmaf(X[1], s.y, fmaf(X[2], s.z, X[3])));
        w.y = fmaf(X[4], s.x, fmaf(X[5], s.y, fmaf(X[6], s.z, X[7])));
        w.z = fmaf(X[8], s.x, fmaf(X[9], s.y, fmaf(X[10], s.z, X[11])));
        w.w = s.w;
        P[a] = w;
      }
      __syncwarp();
      if (!C.ffc) {
        bool hit = false;
        if (C.check_env) {
          for (int a = lane; a < M; a += kWarp) {
            const float4 pa = P[a];
            for (int o = 0; o < C.env_ns; ++o) {
              if (CLR) minclr = fminf(minclr, sph_clr(pa, C.env_s[o]));
              else hit |= sph_hit(pa, C.env_s[o]);
            }
            for (int o = 0; o < C.env_nb; ++o) {
              const float d2 = box_d2(pa, C.env_b + 6 * o);
              if (CLR) minclr = fminf(minclr, sqrtf(d2) - pa.w);
              else hit |= d2 < pa.w * pa.w;
            }
          }
          for (int r = 0; r < n; ++r) {
            const int ns = S.rs[r].n_self;
            const int2 *sp = S.rs[r].self;
            const float4 *Pr = P + S.off[r];
            for (int p = lane; p < ns; p += kWarp) {
              const int2 e = sp[p];
              if (CLR) minclr = fminf(minclr, sph_clr(Pr[e.x], Pr[e.y]));
              else hit |= sph_hit(Pr[e.x], Pr[e.y]);
            }
          }
          C.tests += (unsigned long long)C.envtests;
          // combined order (Alg. 1): env + self of every robot, then pairs
          if (!CLR && !C.exhaustive && __any_sync(0xffffffffu, hit)) return 1;
        }
        for (int a = lane; a < rows; a += kWarp) {
          int r = 0;
          while (a >= S.off[r + 1]) ++r;
          const float4 pa = P[a];
#pragma unroll 4
          for (int bb = S.off[r + 1]; bb < M; ++bb) {
            if (CLR) minclr = fminf(minclr, sph_clr(pa, P[bb]));
            else hit |= sph_hit(pa, P[bb]);
          }
        }
        C.tests += (unsigned long long)C.pairtests;
        if (CLR) hit = minclr < 0.f;
        if (__any_sync(0xffffffffu, hit)) {
          if (!C.exhaustive) return 1;
          found = 1;
        }
      } else {
        unsigned pm = 0;
        for (int a = lane; a < rows; a += kWarp) {
          int r = 0;
          while (a >= S.off[r + 1]) ++r;
          const float4 pa = P[a];
          for (int j = r + 1; j < n; ++j) {
            bool h = false;
#pragma unroll 4
            for (int bb = S.off[j]; bb < S.off[j + 1]; ++bb) h |= sph_hit(pa, P[bb]);
            if (h) pm |= 1u << pair_index(r, j, n);
          }
        }
        C.tests += (unsigned long long)C.pairtests;
        pm = __reduce_or_sync(0xffffffffu, pm);
        if (pm) {
          const int key = t * 32 + (__ffs(pm) - 1);
          if (!C.exhaustive) return key;
          if (key < found) found = key;   // states run in increasing t
        }
      }
      __syncwarp();
    }
    __syncwarp();
  }
  return found;
}

// ---------------------------------------------------------------------------
// the persistent work-stealing kernel
// ---------------------------------------------------------------------------

template <bool CLR>
__device__ void run_chunk(const BatchDev &B, WarpSmem &S, int q, int c, int lane) {
  const QueryDev Q = B.q[q];
  TileCtx C;
  C.q = q; C.T = Q.T; C.n = Q.n; C.M = Q.M; C.nb = Q.ntiles;
  C.ffc = Q.bits & 1u;
  C.check_env = (!C.ffc) && (B.flags & MRV_CHECK_ENV);
  C.exhaustive = (B.flags & MRV_EXHAUSTIVE) ? 1 : 0;
  C.env_ns = 0; C.env_nb = 0; C.env_s = nullptr; C.env_b = nullptr;
  if (C.check_env && Q.env >= 0) {
    const EnvDev &E = B.envs[Q.env];
    C.env_ns = E.n_spheres; C.env_nb = E.n_aabbs; C.env_s = E.spheres; C.env_b = E.aabbs;
  }
  C.pairtests = Q.pairtests; C.envtests = Q.envtests;
  C.tests = 0; C.states = 0;
  // stage the query's robots
  const int s0 = B.q_robot_off[q];
  if (lane < C.n) {
    const int id = B.slot_robot_id[s0 + lane];
    const ModelDev &m = B.models[id];
    RobotSlot rs;
    rs.spheres = m.spheres; rs.links = m.sphere_link; rs.self = m.self_pairs;
    rs.mdl = id; rs.m = m.n_spheres; rs.dof = m.dof; rs.kind = m.kind; rs.n_self = m.n_self;
    rs.w0 = B.slot_wp_off[s0 + lane]; rs.w1 = B.slot_wp_off[s0 + lane + 1]; rs.pad = 0;
    S.rs[lane] = rs;
  }
  __syncwarp();
  if (lane == 0) {
    int acc = 0;
    S.off[0] = 0;
    for (int r = 0; r < C.n; ++r) { acc += S.rs[r].m; S.off[r + 1] = acc; }
  }
  __syncwarp();
  const int b0 = c * Q.cte;
  const int b1 = min(b0 + Q.cte, Q.ntiles);
  float minclr = INFINITY;
  for (int b = b0; b < b1; ++b) {
    if (!C.exhaustive) {
      // one lane reads the query's shared verdict so the warp decides together
      int stop = 0;
      if (lane == 0)
        stop = !C.ffc ? *(volatile int *)&B.q_hit[q] != 0 : *(volatile int *)&B.q_best[q] < b * kWarp * 32;
      if (__shfl_sync(0xffffffffu, stop, 0)) break;
    }
    int res = (Q.bits & 2u) ? tile_flavor_a<CLR>(B, C, S, b, lane, minclr)
                            : tile_flavor_b<CLR>(B, C, S, b, lane, minclr);
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
  if (CLR) {
    for (int o = 16; o > 0; o >>= 1) minclr = fminf(minclr, __shfl_xor_sync(0xffffffffu, minclr, o));
    if (lane == 0) atomicMin((int *)&B.q_minclr[q], f2ord(minclr));
  }
  if (lane == 0) {
    atomicAdd(&B.stats[0], C.states);
    atomicAdd(&B.stats[1], C.tests);
  }
  __syncwarp();
}

template <bool CLR>
__global__ void k_main(BatchDev B, int q_lo, int q_hi) {
  extern __shared__ float4 smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  WarpSmem &S = *reinterpret_cast<WarpSmem *>(reinterpret_cast<char *>(smem_raw) + warp * warp_smem_bytes());
  const long long t_start = clock64();
  if (q_lo >= 0) {
    // single-query mode (one launch per query): block x = chunk x of q_lo
    const QueryDev Q = B.q[q_lo];
    for (int c = blockIdx.x * (blockDim.x >> 5) + warp; c < Q.nchunks; c += gridDim.x * (blockDim.x >> 5))
      if (!(Q.bits & 4u)) run_chunk<CLR>(B, S, q_lo, c, lane);
    return;
  }
  const int n_items = B.counters[1];
  unsigned long long items = 0;
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(&B.counters[0], 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= n_items) break;
    int halt = 0;
    if (lane == 0) {
      if (*(volatile int *)&B.counters[2]) halt = 1;
      else if (B.clock_budget > 0 && clock64() - t_start > B.clock_budget) halt = 2;
      if (halt) atomicOr(B.err, halt == 1 ? kErrAbort : kErrTimeout);
    }
    if (__shfl_sync(0xffffffffu, halt, 0)) break;
    int lo = 0, hi = kMaxLevels - 1;   // level: last c with level_start[c] <= idx
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (B.level_start[mid] <= idx) lo = mid;
      else hi = mid - 1;
    }
    const int q = B.sorted[idx - B.level_start[lo]];
    run_chunk<CLR>(B, S, q, lo, lane);
    ++items;
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
      c.t = key >> 5;
      int p = key & 31, i = 0;
      while (p >= Q.n - 1 - i) { p -= Q.n - 1 - i; ++i; }
      c.i = i;
      c.j = i + 1 + p;
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
    r.spheres = m.spheres; r.links = m.sphere_link; r.self = m.self_pairs;
    r.mdl = id; r.m = m.n_spheres; r.dof = m.dof; r.kind = m.kind; r.n_self = m.n_self;
    r.w0 = B.slot_wp_off[s0 + threadIdx.x]; r.w1 = B.slot_wp_off[s0 + threadIdx.x + 1]; r.pad = 0;
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
    const float *X = xf + r * kMaxLinks * 12 + rs[r].links[i] * 12;
    P[a] = make_float4(fmaf(X[0], s.x, fmaf(X[1], s.y, fmaf(X[2], s.z, X[3]))),
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
        for (int o = 0; o < E->n_aabbs; ++o) m = fminf(m, sqrtf(box_d2(pa, E->aabbs + 6 * o)) - pa.w);
      }
      const int li = a - off[r];
      for (int p = 0; p < rs[r].n_self; ++p) {
        const int2 e = rs[r].self[p];
        if (e.x == li) m = fminf(m, sph_clr(pa, P[off[r] + e.y]));
        else if (e.y == li) m = fminf(m, sph_clr(pa, P[off[r] + e.x]));
      }
    }
    out[(size_t)k * Q.M + a] = m;
  }
}

// ---------------------------------------------------------------------------
// host-side launch wrappers
// ---------------------------------------------------------------------------

size_t main_smem_bytes(int warps) { return warp_smem_bytes() * (size_t)warps; }

cudaError_t launch_prepare(const BatchDev &B, cudaStream_t st) {
  if (B.n_queries > 0) {
    const int th = 128, bl = (B.n_queries + th - 1) / th;
    k_prep<<<bl, th, 0, st>>>(B);
  }
  k_levels<<<1, 32, 0, st>>>(B);
  if (B.n_queries > 0) {
    const int th = 256, bl = (B.n_queries + th - 1) / th;
    k_scatter<<<bl, th, 0, st>>>(B);
  }
  return cudaGetLastError();
}

cudaError_t set_main_attrs(int warps) {
  const int bytes = (int)main_smem_bytes(warps);
  cudaError_t e = cudaFuncSetAttribute(k_main<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_main<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t max_blocks_per_sm(int warps, bool clr, int *out) {
  set_main_attrs(warps);
  if (clr)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_main<true>, warps * 32, main_smem_bytes(warps));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_main<false>, warps * 32, main_smem_bytes(warps));
}

cudaError_t launch_main(const BatchDev &B, int grid, int warps, bool clr, int q_single, cudaStream_t st) {
  const size_t smem = main_smem_bytes(warps);
  if (clr) k_main<true><<<grid, warps * 32, smem, st>>>(B, q_single, q_single);
  else k_main<false><<<grid, warps * 32, smem, st>>>(B, q_single, q_single);
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
