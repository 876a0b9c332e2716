/*
 * FP64 scalar oracle for multi-robot MotionValidation (MV) and
 * FindFirstConflict (FFC).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it reads the same FP32 input
 * arrays and promotes every value to double.
 *
 * What it computes is the plain definition of the two primitives, written as
 * exhaustive loops in natural order (timestep, then robot, then robot pair,
 * then sphere pair).  Early return is used only where it cannot change the
 * answer.  The paper's batch packing (rake / linear, Sec. III-A, Fig. 2) and
 * its combined / hierarchical orders only change how much work is done, not
 * the answer (Sec. III-A, Sec. IV-B), so none of them appears here.
 *
 * Definitions followed (paper sections):
 *   - states: each robot moves at most `resolution` C-space units (Euclidean,
 *     unweighted) per timestep; a composite motion takes the longest robot's
 *     step count and time-scales the others to start and end together
 *     (Sec. IV-A3).  Timed waypoint paths are interpolated linearly per
 *     segment; a path shorter than the composite one is padded with its last
 *     configuration (Sec. III-A, PackCfgBatch note).
 *   - SpheresFK: robot configuration -> world sphere centers through the
 *     kinematic chain (Sec. II-B, Sec. III-A); modified (Craig) DH is used:
 *       X_k = X_{k-1} RotX(alpha_k) TransX(a_k) RotZ(theta_k + q_k) TransZ(d_k).
 *   - CC: robot vs obstacle spheres, boxes and cylinders and robot self-collision
 *     (Alg. 1, robot-obstacle step), robot vs robot sphere sets (Alg. 1,
 *     robot-robot step; Alg. 2).  Collision iff clearance < 0 with
 *       sphere-sphere clearance = |c_a - c_b| - r_a - r_b,
 *       sphere-box clearance    = dist(c, box) - r   (dist = 0 inside),
 *       sphere-cylinder clearance = dist(c, cylinder) - r (solid, flat caps;
 *       the obstacle kind of the paper's Cage scenario, Sec. V-A).
 *   - MV (Alg. 1): invalid iff some state has an env/self collision (when
 *     check_environment is set) or a robot-robot collision.
 *   - FFC (Alg. 2): the lexicographically smallest (t, i, j), i < j, with
 *     robots i and j colliding at t; no obstacle or self checks.
 *
 * Decidability margins (the FP32 GPU result is compared exactly only where
 * the FP64 clearance keeps away from zero) and the per-sphere clearance
 * diagnostic are defined alongside.
 *
 * All functions return 0 on success and a negative code on malformed input.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_DOF 16
#define ORC_MAX_ROBOTS 64
#define ORC_MAX_LINKS (ORC_MAX_DOF + 2)

typedef struct {
  int32_t kind;          /* 0: modified-DH chain, 1: point robot          */
  int32_t dof;
  const float *dh;       /* dof x 4: a, alpha, d, theta_offset            */
  const float *flange;   /* 3x4 or NULL (identity)                        */
  const float *base;     /* 3x4 world <- base                             */
  float point_z;         /* point robot, dof 2: fixed z                   */
  int32_t n_spheres;
  const int32_t *sphere_link;
  const float *sphere_xyzr;
  int32_t n_self;
  const int32_t *self_pairs; /* n_self x 2 sphere indices                 */
} orc_robot;

typedef struct {
  int32_t n_spheres;
  const float *spheres;  /* n x 4 */
  int32_t n_aabbs;
  const float *aabbs;    /* n x 6: lo xyz, hi xyz */
  int32_t n_cylinders;
  const float *cylinders; /* n x 7: axis end a xyz, axis end b xyz, radius */
} orc_env;

typedef struct {
  int32_t n_queries;
  const int32_t *q_robot_off;
  const int32_t *slot_robot;   /* index into the robot array */
  const int32_t *slot_wp_off;
  const float *waypoints;      /* wp_stride floats per waypoint */
  int32_t wp_stride;
  const int32_t *seg_steps;    /* per waypoint, or NULL: start/goal form */
  double resolution;
} orc_batch;

/* ------------------------------------------------------------------------ */
/* 4x4 homogeneous matrices                                                  */
/* ------------------------------------------------------------------------ */

typedef struct { double m[4][4]; } mat4;

static mat4 mat_identity(void) {
  mat4 r;
  memset(&r, 0, sizeof r);
  for (int i = 0; i < 4; ++i) r.m[i][i] = 1.0;
  return r;
}

static mat4 mat_mul(const mat4 *a, const mat4 *b) {
  mat4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a->m[i][k] * b->m[k][j];
      r.m[i][j] = s;
    }
  return r;
}

static mat4 mat_from34(const float *p) {
  mat4 r = mat_identity();
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) r.m[i][j] = (double)p[i * 4 + j];
  return r;
}

static mat4 rot_x(double a) {
  mat4 r = mat_identity();
  r.m[1][1] = cos(a); r.m[1][2] = -sin(a);
  r.m[2][1] = sin(a); r.m[2][2] = cos(a);
  return r;
}

static mat4 rot_z(double a) {
  mat4 r = mat_identity();
  r.m[0][0] = cos(a); r.m[0][1] = -sin(a);
  r.m[1][0] = sin(a); r.m[1][1] = cos(a);
  return r;
}

static mat4 trans(double x, double y, double z) {
  mat4 r = mat_identity();
  r.m[0][3] = x; r.m[1][3] = y; r.m[2][3] = z;
  return r;
}

/* One modified-DH joint: RotX(alpha) TransX(a) RotZ(theta) TransZ(d). */
static mat4 dh_joint(double a, double alpha, double d, double theta) {
  mat4 rx = rot_x(alpha), tx = trans(a, 0, 0), rz = rot_z(theta), tz = trans(0, 0, d);
  mat4 t1 = mat_mul(&rx, &tx);
  mat4 t2 = mat_mul(&t1, &rz);
  return mat_mul(&t2, &tz);
}

/* ------------------------------------------------------------------------ */
/* SpheresFK (Sec. II-B, Sec. III-A)                                         */
/* ------------------------------------------------------------------------ */

/* World sphere centers of robot `r` at configuration q (dof doubles).
 * centers: n_spheres x 3. */
int orc_fk(const orc_robot *r, const double *q, double *centers) {
  if (r->dof < 0 || r->dof > ORC_MAX_DOF) return -1;
  mat4 frame[ORC_MAX_LINKS];
  int n_frames;
  frame[0] = mat_from34(r->base);
  if (r->kind == 0) {
    for (int k = 1; k <= r->dof; ++k) {
      const float *row = r->dh + 4 * (k - 1);
      mat4 j = dh_joint(row[0], row[1], row[2], (double)row[3] + q[k - 1]);
      frame[k] = mat_mul(&frame[k - 1], &j);
    }
    mat4 fl = r->flange ? mat_from34(r->flange) : mat_identity();
    frame[r->dof + 1] = mat_mul(&frame[r->dof], &fl);
    n_frames = r->dof + 2;
  } else if (r->kind == 1) {
    if (r->dof != 2 && r->dof != 3) return -1;
    double z = r->dof == 2 ? (double)r->point_z : q[2];
    mat4 t = trans(q[0], q[1], z);
    frame[1] = mat_mul(&frame[0], &t);
    n_frames = 2;
  } else {
    return -1;
  }
  for (int s = 0; s < r->n_spheres; ++s) {
    int l = r->sphere_link[s];
    if (l < 0 || l >= n_frames) return -2;
    const float *c = r->sphere_xyzr + 4 * s;
    for (int i = 0; i < 3; ++i)
      centers[3 * s + i] = frame[l].m[i][0] * c[0] + frame[l].m[i][1] * c[1] +
                           frame[l].m[i][2] * c[2] + frame[l].m[i][3];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* clearances (CC, Sec. III-A)                                               */
/* ------------------------------------------------------------------------ */

double orc_sphere_sphere(const double *ca, double ra, const double *cb, double rb) {
  double dx = ca[0] - cb[0], dy = ca[1] - cb[1], dz = ca[2] - cb[2];
  return sqrt(dx * dx + dy * dy + dz * dz) - ra - rb;
}

double orc_sphere_box(const double *c, double r, const float *box) {
  double s = 0.0;
  for (int i = 0; i < 3; ++i) {
    double lo = box[i], hi = box[3 + i], e = 0.0;
    if (c[i] < lo) e = lo - c[i];
    else if (c[i] > hi) e = c[i] - hi;
    s += e * e;
  }
  return sqrt(s) - r;
}

/* Signed clearance between a sphere and a solid finite cylinder with flat
 * caps, axis from a to b, radius rho: distance from the center to the solid
 * (0 inside) minus r.  With s the center's coordinate along the unit axis
 * from a and d its distance from the axis line, the nearest point of the
 * solid clamps s to [0, L] and d to [0, rho], so the distance is
 * sqrt(excess(s)^2 + excess(d)^2). */
double orc_sphere_cylinder(const double *c, double r, const float *cyl) {
  double u[3], w[3], L = 0.0;
  for (int k = 0; k < 3; ++k) {
    u[k] = (double)cyl[3 + k] - (double)cyl[k];
    w[k] = c[k] - (double)cyl[k];
    L += u[k] * u[k];
  }
  L = sqrt(L);
  for (int k = 0; k < 3; ++k) u[k] /= L;
  const double s = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
  double d2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double p = w[k] - s * u[k];
    d2 += p * p;
  }
  const double d = sqrt(d2), rho = cyl[6];
  const double es = s < 0.0 ? -s : (s > L ? s - L : 0.0);
  const double ed = d > rho ? d - rho : 0.0;
  return sqrt(es * es + ed * ed) - r;
}

/* ------------------------------------------------------------------------ */
/* discretisation (Sec. IV-A3) and padding (Sec. III-A)                      */
/* ------------------------------------------------------------------------ */

/* Step count of a start->goal motion: ceil(|g - s|_2 / resolution), 0 when
 * the robot does not move.  Summation runs over the joints in index order
 * and every operation is a separately rounded IEEE double operation. */
static int64_t steps_for(const float *s, const float *g, int dof, double res) {
  double acc = 0.0;
  for (int k = 0; k < dof; ++k) {
    double d = (double)g[k] - (double)s[k];
    acc = acc + d * d;
  }
  double dist = sqrt(acc);
  if (dist == 0.0) return 0;
  return (int64_t)ceil(dist / res);
}

/* Composite step count T of query q (states 0..T). */
int orc_query_T(const orc_batch *b, const orc_robot *robots, int q, int64_t *T_out) {
  int s0 = b->q_robot_off[q], s1 = b->q_robot_off[q + 1];
  int64_t T = 0;
  for (int s = s0; s < s1; ++s) {
    int w0 = b->slot_wp_off[s], w1 = b->slot_wp_off[s + 1];
    if (w1 <= w0) return -1;
    const orc_robot *r = &robots[b->slot_robot[s]];
    int64_t Ts = 0;
    if (b->seg_steps == NULL) {
      if (w1 - w0 != 2) return -1;
      Ts = steps_for(b->waypoints + (size_t)w0 * b->wp_stride,
                     b->waypoints + (size_t)(w0 + 1) * b->wp_stride, r->dof, b->resolution);
    } else {
      for (int w = w0; w < w1 - 1; ++w) {
        if (b->seg_steps[w] < 0) return -1;
        Ts += b->seg_steps[w];
      }
    }
    if (Ts > T) T = Ts;
  }
  *T_out = T;
  return 0;
}

/* Configuration of slot s at timestep t of its query (composite step count
 * T).  q_out: dof doubles. */
static void slot_state(const orc_batch *b, const orc_robot *robots, int s, int64_t T, int64_t t,
                       double *q_out) {
  int w0 = b->slot_wp_off[s], w1 = b->slot_wp_off[s + 1];
  int dof = robots[b->slot_robot[s]].dof;
  const float *W = b->waypoints;
  size_t st = (size_t)b->wp_stride;
  if (b->seg_steps == NULL) {
    /* start/goal form: every robot of the query is time-scaled to T steps */
    const float *a = W + (size_t)w0 * st, *g = W + (size_t)(w0 + 1) * st;
    for (int k = 0; k < dof; ++k) {
      if (T == 0) q_out[k] = (double)a[k];
      else q_out[k] = (double)a[k] + ((double)g[k] - (double)a[k]) * ((double)t / (double)T);
    }
    return;
  }
  int64_t tau = 0;
  for (int w = w0; w < w1 - 1; ++w) {
    int64_t n = b->seg_steps[w];
    if (t < tau + n) {
      const float *a = W + (size_t)w * st, *g = W + (size_t)(w + 1) * st;
      double f = (double)(t - tau) / (double)n;
      for (int k = 0; k < dof; ++k) q_out[k] = (double)a[k] + ((double)g[k] - (double)a[k]) * f;
      return;
    }
    tau += n;
  }
  /* at or past the end of this slot's path: hold the last configuration */
  const float *l = W + (size_t)(w1 - 1) * st;
  for (int k = 0; k < dof; ++k) q_out[k] = (double)l[k];
}

/* ------------------------------------------------------------------------ */
/* per-state geometry of one query                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n;                     /* robots in the query           */
  const orc_robot *r[ORC_MAX_ROBOTS];
  int off[ORC_MAX_ROBOTS + 1];  /* sphere offsets per robot   */
  double *c;                 /* total spheres x 3             */
} qstate;

static int qstate_init(qstate *qs, const orc_batch *b, const orc_robot *robots, int q) {
  int s0 = b->q_robot_off[q], s1 = b->q_robot_off[q + 1];
  qs->n = s1 - s0;
  if (qs->n < 0 || qs->n > ORC_MAX_ROBOTS) return -1;
  qs->off[0] = 0;
  for (int i = 0; i < qs->n; ++i) {
    qs->r[i] = &robots[b->slot_robot[s0 + i]];
    qs->off[i + 1] = qs->off[i] + qs->r[i]->n_spheres;
  }
  qs->c = (double *)malloc(sizeof(double) * 3 * (size_t)(qs->off[qs->n] > 0 ? qs->off[qs->n] : 1));
  return qs->c ? 0 : -3;
}

static void qstate_free(qstate *qs) { free(qs->c); }

static int qstate_fk(qstate *qs, const orc_batch *b, const orc_robot *robots, int q, int64_t T,
                     int64_t t) {
  double cfg[ORC_MAX_DOF];
  int s0 = b->q_robot_off[q];
  for (int i = 0; i < qs->n; ++i) {
    slot_state(b, robots, s0 + i, T, t, cfg);
    if (orc_fk(qs->r[i], cfg, qs->c + 3 * (size_t)qs->off[i]) != 0) return -2;
  }
  return 0;
}

/* min clearance of robot i against the environment and itself */
static double env_self_min(const qstate *qs, const orc_env *e, int i) {
  double m = INFINITY;
  const orc_robot *r = qs->r[i];
  const double *C = qs->c + 3 * (size_t)qs->off[i];
  for (int a = 0; a < r->n_spheres; ++a) {
    double ra = r->sphere_xyzr[4 * a + 3];
    if (e) {
      for (int o = 0; o < e->n_spheres; ++o) {
        double co[3] = {e->spheres[4 * o], e->spheres[4 * o + 1], e->spheres[4 * o + 2]};
        double v = orc_sphere_sphere(C + 3 * a, ra, co, e->spheres[4 * o + 3]);
        if (v < m) m = v;
      }
      for (int o = 0; o < e->n_aabbs; ++o) {
        double v = orc_sphere_box(C + 3 * a, ra, e->aabbs + 6 * o);
        if (v < m) m = v;
      }
      for (int o = 0; o < e->n_cylinders; ++o) {
        double v = orc_sphere_cylinder(C + 3 * a, ra, e->cylinders + 7 * o);
        if (v < m) m = v;
      }
    }
  }
  for (int p = 0; p < r->n_self; ++p) {
    int a = r->self_pairs[2 * p], c = r->self_pairs[2 * p + 1];
    double v = orc_sphere_sphere(C + 3 * a, r->sphere_xyzr[4 * a + 3], C + 3 * c,
                                 r->sphere_xyzr[4 * c + 3]);
    if (v < m) m = v;
  }
  return m;
}

/* min clearance between robots i and j */
static double pair_min(const qstate *qs, int i, int j) {
  double m = INFINITY;
  const orc_robot *ri = qs->r[i], *rj = qs->r[j];
  const double *Ci = qs->c + 3 * (size_t)qs->off[i], *Cj = qs->c + 3 * (size_t)qs->off[j];
  for (int a = 0; a < ri->n_spheres; ++a)
    for (int c = 0; c < rj->n_spheres; ++c) {
      double v = orc_sphere_sphere(Ci + 3 * a, ri->sphere_xyzr[4 * a + 3], Cj + 3 * c,
                                   rj->sphere_xyzr[4 * c + 3]);
      if (v < m) m = v;
    }
  return m;
}

static int check_self_pairs(const orc_robot *r) {
  for (int p = 0; p < r->n_self; ++p) {
    int a = r->self_pairs[2 * p], c = r->self_pairs[2 * p + 1];
    if (a < 0 || c < 0 || a >= r->n_spheres || c >= r->n_spheres) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* MV (Alg. 1) — plain definition                                            */
/* ------------------------------------------------------------------------ */

/* valid_out = 1 iff no state of query q has a collision.  env may be NULL
 * (no obstacles); self-collision pairs are checked only when check_env is
 * set (robot-obstacle validation includes self-collision, Sec. III-A). */
int orc_mv(const orc_batch *b, const orc_robot *robots, const orc_env *env, int check_env, int q,
           int *valid_out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  for (int i = 0; i < qs.n; ++i)
    if (check_self_pairs(qs.r[i])) { qstate_free(&qs); return -1; }
  int valid = 1, rc = 0;
  for (int64_t t = 0; t <= T && valid; ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    if (check_env)
      for (int i = 0; i < qs.n && valid; ++i)
        if (env_self_min(&qs, env, i) < 0.0) valid = 0;
    for (int i = 0; i < qs.n && valid; ++i)
      for (int j = i + 1; j < qs.n && valid; ++j)
        if (pair_min(&qs, i, j) < 0.0) valid = 0;
  }
  qstate_free(&qs);
  *valid_out = valid;
  return rc;
}

/* Signed minimum clearance over every check MV performs for query q.  The
 * scan stops as soon as the running minimum falls below `stop_below` (pass
 * -INFINITY for the full minimum). */
int orc_mv_min_clearance(const orc_batch *b, const orc_robot *robots, const orc_env *env,
                         int check_env, int q, double stop_below, double *out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  for (int i = 0; i < qs.n; ++i)
    if (check_self_pairs(qs.r[i])) { qstate_free(&qs); return -1; }
  double m = INFINITY;
  int rc = 0;
  for (int64_t t = 0; t <= T && !(m < stop_below); ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    if (check_env)
      for (int i = 0; i < qs.n; ++i) {
        double v = env_self_min(&qs, env, i);
        if (v < m) m = v;
      }
    for (int i = 0; i < qs.n; ++i)
      for (int j = i + 1; j < qs.n; ++j) {
        double v = pair_min(&qs, i, j);
        if (v < m) m = v;
      }
  }
  qstate_free(&qs);
  *out = m;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* MV of prioritized planning (PP-ST-RRT, Sec. IV-C) — plain definition      */
/* ------------------------------------------------------------------------ */

/* The planner validates one robot at a time against the paths of the robots
 * planned before it, which act as moving obstacles (Sec. IV-C, PP-ST-RRT):
 * Alg. 1's loop over robots for the obstacle and self checks keeps only the
 * current robot, and its robot-robot loop keeps only the pairs of the current
 * robot with the higher-priority ones.  Slot 0 of the query is the current
 * robot, slots 1..n-1 the higher-priority robots.  valid_out = 1 iff no state
 * has a collision of robot 0 with the obstacles or itself (check_env) or with
 * any robot j >= 1.  Collisions among the higher-priority robots, and theirs
 * with the obstacles, are not part of the check. */
int orc_mv_prio(const orc_batch *b, const orc_robot *robots, const orc_env *env, int check_env, int q,
                int *valid_out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  for (int i = 0; i < qs.n; ++i)
    if (check_self_pairs(qs.r[i])) { qstate_free(&qs); return -1; }
  int valid = 1, rc = 0;
  for (int64_t t = 0; valid && t <= T; ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    if (check_env && env_self_min(&qs, env, 0) < 0.0) valid = 0;
    for (int j = 1; j < qs.n && valid; ++j)
      if (pair_min(&qs, 0, j) < 0.0) valid = 0;
  }
  qstate_free(&qs);
  *valid_out = valid;
  return rc;
}

/* Signed minimum clearance over the checks of orc_mv_prio (scan stops once
 * the running minimum falls below stop_below). */
int orc_mv_prio_min_clearance(const orc_batch *b, const orc_robot *robots, const orc_env *env,
                              int check_env, int q, double stop_below, double *out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  for (int i = 0; i < qs.n; ++i)
    if (check_self_pairs(qs.r[i])) { qstate_free(&qs); return -1; }
  double m = INFINITY;
  int rc = 0;
  for (int64_t t = 0; t <= T && !(m < stop_below); ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    if (check_env) {
      double v = env_self_min(&qs, env, 0);
      if (v < m) m = v;
    }
    for (int j = 1; j < qs.n; ++j) {
      double v = pair_min(&qs, 0, j);
      if (v < m) m = v;
    }
  }
  qstate_free(&qs);
  *out = m;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* FFC (Alg. 2) — plain definition                                           */
/* ------------------------------------------------------------------------ */

/* out3 = (t, i, j): the lexicographically smallest colliding (t, i<j), or
 * (-1, -1, -1).  i, j are 0-based slot positions inside the query. */
int orc_ffc(const orc_batch *b, const orc_robot *robots, int q, int32_t *out3) {
  int64_t T;
  out3[0] = out3[1] = out3[2] = -1;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  int rc = 0, found = 0;
  for (int64_t t = 0; t <= T && !found; ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    for (int i = 0; i < qs.n && !found; ++i)
      for (int j = i + 1; j < qs.n && !found; ++j)
        if (pair_min(&qs, i, j) < 0.0) {
          out3[0] = (int32_t)t; out3[1] = i; out3[2] = j;
          found = 1;
        }
  }
  qstate_free(&qs);
  return rc;
}

/* The first conflict deeper than a bound: the lexicographically smallest
 * (t, i, j), i < j, whose pair clearance is below `bound` (Alg. 2's order
 * with the collision test `clearance < 0` replaced by `clearance < bound`),
 * or (-1, -1, -1).  With bound = -margin it is the first pair that every
 * correct FP32 answer must not skip: an answer later than it passed over a
 * collision deeper than the decidability margin. */
int orc_ffc_below(const orc_batch *b, const orc_robot *robots, int q, double bound, int32_t *out3) {
  int64_t T;
  out3[0] = out3[1] = out3[2] = -1;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  int rc = 0, found = 0;
  for (int64_t t = 0; !found && t <= T; ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    for (int i = 0; i < qs.n && !found; ++i)
      for (int j = i + 1; j < qs.n && !found; ++j)
        if (pair_min(&qs, i, j) < bound) {
          out3[0] = (int32_t)t; out3[1] = i; out3[2] = j;
          found = 1;
        }
  }
  qstate_free(&qs);
  return rc;
}

/* FFC decidability: 1 iff every robot pair visited before the answer (in
 * (t, i, j) order) has clearance > margin and the answer's pair has
 * clearance < -margin (no answer: every pair at every state > margin). */
int orc_ffc_decidable(const orc_batch *b, const orc_robot *robots, int q, double margin,
                      int *decidable_out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  int rc = 0, done = 0, dec = 1;
  for (int64_t t = 0; t <= T && !done; ++t) {
    if ((rc = qstate_fk(&qs, b, robots, q, T, t))) break;
    for (int i = 0; i < qs.n && !done; ++i)
      for (int j = i + 1; j < qs.n && !done; ++j) {
        double v = pair_min(&qs, i, j);
        if (v < 0.0) {
          done = 1;
          if (!(v < -margin)) dec = 0;
        } else if (!(v > margin)) {
          dec = 0;
        }
      }
  }
  qstate_free(&qs);
  *decidable_out = dec;
  return rc;
}

/* Pairwise minimum clearance of every robot pair at state t (n*(n-1)/2
 * values in (i, j) lexicographic order). */
int orc_pair_clearances(const orc_batch *b, const orc_robot *robots, int q, int64_t t,
                        double *out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  int rc = qstate_fk(&qs, b, robots, q, T, t), k = 0;
  if (!rc)
    for (int i = 0; i < qs.n; ++i)
      for (int j = i + 1; j < qs.n; ++j) out[k++] = pair_min(&qs, i, j);
  qstate_free(&qs);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* per-sphere clearance diagnostic                                           */
/* ------------------------------------------------------------------------ */

/* For each listed timestep and each sphere of the query (robots in slot
 * order, spheres in model order): the minimum clearance over the checks that
 * involve that sphere — other robots' spheres always, obstacles and listed
 * self pairs when check_env is set.  +inf when no check involves it.
 * out: nt x total_spheres. */
int orc_clearance(const orc_batch *b, const orc_robot *robots, const orc_env *env, int check_env,
                  int q, const int64_t *ts, int nt, double *out) {
  int64_t T;
  if (orc_query_T(b, robots, q, &T)) return -1;
  qstate qs;
  if (qstate_init(&qs, b, robots, q)) return -1;
  int M = qs.off[qs.n], rc = 0;
  for (int k = 0; k < nt && !rc; ++k) {
    double *o = out + (size_t)k * M;
    for (int a = 0; a < M; ++a) o[a] = INFINITY;
    if (ts[k] < 0 || ts[k] > T) { rc = -1; break; }
    if ((rc = qstate_fk(&qs, b, robots, q, T, ts[k]))) break;
    for (int i = 0; i < qs.n; ++i) {
      const orc_robot *ri = qs.r[i];
      for (int a = 0; a < ri->n_spheres; ++a) {
        const double *ca = qs.c + 3 * (size_t)(qs.off[i] + a);
        double ra = ri->sphere_xyzr[4 * a + 3], m = INFINITY;
        for (int j = 0; j < qs.n; ++j) {
          if (j == i) continue;
          const orc_robot *rj = qs.r[j];
          for (int c = 0; c < rj->n_spheres; ++c) {
            double v = orc_sphere_sphere(ca, ra, qs.c + 3 * (size_t)(qs.off[j] + c),
                                         rj->sphere_xyzr[4 * c + 3]);
            if (v < m) m = v;
          }
        }
        if (check_env) {
          if (env) {
            for (int s = 0; s < env->n_spheres; ++s) {
              double co[3] = {env->spheres[4 * s], env->spheres[4 * s + 1], env->spheres[4 * s + 2]};
              double v = orc_sphere_sphere(ca, ra, co, env->spheres[4 * s + 3]);
              if (v < m) m = v;
            }
            for (int s = 0; s < env->n_aabbs; ++s) {
              double v = orc_sphere_box(ca, ra, env->aabbs + 6 * s);
              if (v < m) m = v;
            }
            for (int s = 0; s < env->n_cylinders; ++s) {
              double v = orc_sphere_cylinder(ca, ra, env->cylinders + 7 * s);
              if (v < m) m = v;
            }
          }
          for (int p = 0; p < ri->n_self; ++p) {
            int x = ri->self_pairs[2 * p], y = ri->self_pairs[2 * p + 1];
            if (x != a && y != a) continue;
            int other = x == a ? y : x;
            double v = orc_sphere_sphere(ca, ra, qs.c + 3 * (size_t)(qs.off[i] + other),
                                         ri->sphere_xyzr[4 * other + 3]);
            if (v < m) m = v;
          }
        }
        o[qs.off[i] + a] = m;
      }
    }
  }
  qstate_free(&qs);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* batch drivers (independent queries, static interleaved partition)         */
/* ------------------------------------------------------------------------ */

enum { JOB_MV, JOB_FFC, JOB_MINCLR, JOB_FFC_DEC, JOB_T, JOB_MV_PRIO, JOB_MINCLR_PRIO, JOB_FFC_BELOW };

typedef struct {
  int job;
  const orc_batch *b;
  const orc_robot *robots;
  const orc_env *const *envs;  /* per query env (may be NULL entries) */
  const int32_t *q_idx;        /* queries to run (NULL: 0..n-1)       */
  int n;
  int check_env;
  double param;
  void *out;
  int tid, nthreads;
  int rc;
} job_t;

static void *job_run(void *arg) {
  job_t *J = (job_t *)arg;
  J->rc = 0;
  for (int k = J->tid; k < J->n; k += J->nthreads) {
    int q = J->q_idx ? J->q_idx[k] : k;
    const orc_env *e = J->envs ? J->envs[k] : NULL;
    int rc = 0;
    switch (J->job) {
      case JOB_MV: {
        int v = 0;
        rc = orc_mv(J->b, J->robots, e, J->check_env, q, &v);
        ((uint8_t *)J->out)[k] = (uint8_t)v;
        break;
      }
      case JOB_FFC:
        rc = orc_ffc(J->b, J->robots, q, (int32_t *)J->out + 3 * (size_t)k);
        break;
      case JOB_MINCLR:
        rc = orc_mv_min_clearance(J->b, J->robots, e, J->check_env, q, J->param,
                                  (double *)J->out + k);
        break;
      case JOB_FFC_DEC: {
        int d = 0;
        rc = orc_ffc_decidable(J->b, J->robots, q, J->param, &d);
        ((uint8_t *)J->out)[k] = (uint8_t)d;
        break;
      }
      case JOB_T:
        rc = orc_query_T(J->b, J->robots, q, (int64_t *)J->out + k);
        break;
      case JOB_MV_PRIO: {
        int v = 0;
        rc = orc_mv_prio(J->b, J->robots, e, J->check_env, q, &v);
        ((uint8_t *)J->out)[k] = (uint8_t)v;
        break;
      }
      case JOB_MINCLR_PRIO:
        rc = orc_mv_prio_min_clearance(J->b, J->robots, e, J->check_env, q, J->param,
                                       (double *)J->out + k);
        break;
      case JOB_FFC_BELOW:
        rc = orc_ffc_below(J->b, J->robots, q, J->param, (int32_t *)J->out + 3 * (size_t)k);
        break;
    }
    if (rc && !J->rc) J->rc = rc;
  }
  return NULL;
}

/* Runs `job` over n queries on nthreads POSIX threads.  envs: per-query env
 * pointers (array of n, entries may be NULL) or NULL for none. */
int orc_batch_run(int job, const orc_batch *b, const orc_robot *robots, const orc_env *const *envs,
                  const int32_t *q_idx, int n, int check_env, double param, void *out,
                  int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  job_t jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (job_t){job, b, robots, envs, q_idx, n, check_env, param, out, t, nthreads, 0};
  }
  if (nthreads == 1) {
    job_run(&jobs[0]);
    return jobs[0].rc;
  }
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, job_run, &jobs[t]) != 0) break;
    ++started;
  }
  for (int t = started; t < nthreads; ++t) job_run(&jobs[t]);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < nthreads; ++t)
    if (jobs[t].rc) return jobs[t].rc;
  return 0;
}
