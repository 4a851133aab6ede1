/*
 * mppi_oracle.c -- plain, slow FP64 CPU restatement of one MPPI solve of the
 * reference-free drone-racing controller (arXiv 2509.14726).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: it is loaded by the tests, by __graft_entry__.smoke() and by
 * the bench's cpu_baseline / reference leg, to check and to time the CUDA path.
 * It shares no source with the CUDA library (its own structs, its own Philox,
 * its own dynamics); the only thing both sides share are the seeded input
 * tables (gates, arc-length path, reference trajectory) built in numpy.
 *
 * Everything is done one sample at a time, one step at a time, in the order
 * the paper states it:
 *   Sec. III-B, Eq. 3 : U^m = U* + dU^m, du ~ N(0, Sigma)
 *   Sec. III-A, Eq. 2 : quadrotor rigid-body model, integrated by RK4
 *   Sec. IV-A, Eq. 6/7: gate progress with per-state gate switching, the
 *                       temporal-consistency pass rule and the near-gate term
 *   Sec. IV-B, Eq. 8  : full-state trajectory tracking
 *   Sec. IV-B, Eq. 9  : contouring against an arc-length parameterised path
 *   Sec. III-B, Eq. 4 : exponential weights
 *   Sec. III-B, Eq. 5 : weighted average -> new nominal, warm start
 *   Algorithm 1       : the loop that ties these together.
 *
 * Readings where the paper is silent (all configurable through or_params):
 *   - input is collective thrust + body-rate command (CTBR); the body-rate
 *     loop is tau = J k_w (w_cmd - w), so dw = k_w (w_cmd - w) - J^-1 (w x Jw)
 *   - Hamilton quaternions, scalar first, R maps body to world, z up,
 *     gravity (0, 0, -g); q is renormalised after every RK4 step
 *   - Philox4x32-10 (Salmon et al., SC'11) with key (seed, drone) and counter
 *     (sample, step, iteration, block); uniforms ((x >> 8) + 1) * 2^-24 in
 *     (0, 1]; Box-Muller turns (x0, x1) and (x2, x3) into four normals;
 *     the 5th (progress) normals of steps 4j .. 4j+3 are the four normals of
 *     block 1 at step 4j, in order
 *   - inputs are clamped to their box; the clamped samples are rolled out and
 *     averaged; the feasibility penalty acts on body rate and altitude
 *   - warm start shifts the new nominal by one step and repeats the last row
 *     (warm_start 0); warm_start 1 keeps the complete sequence, the literal
 *     reading of Sec. III-B;
 *   - nominal_sample 1 makes candidate 0 the unperturbed nominal (Eq. 3 with
 *     du = 0), a common MPPI variant the paper does not use.
 *   - rotor model (kind 1, Eq. 2 as printed): u = dT_s/dt per rotor, held
 *     over the step; the thrusts follow T0 + u t exactly and saturate in
 *     [thrust_min, thrust_max] (Table I: [0, 10] N, rates [-10, 10]); RK4
 *     takes the exact stage thrusts (T is not integrated); l = 0.15 m and
 *     c_tau = 0.01 m (not given); the rotor thrusts at x0 are the
 *     controller's own integrated commands (hover until set); U starts at 0;
 *     tracking weighs the rates themselves, contouring the rotor thrust
 *     changes T_{k+1} - T_k.
 *
 * Parity status: every function here is pinned by a CPU test against a
 * closed form, an invariant, a brute-force search or an independent library
 * (cuRAND's host Philox generator); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NX 13
#define OR_NU 5

/* ---------------------------------------------------------------------- */
/* Parameter blocks (the oracle's own; mirrored by ctypes in oracle.py)    */
/* ---------------------------------------------------------------------- */

typedef struct {
  double mass;        /* kg */
  double inertia[3];  /* diagonal of J, kg m^2 */
  double gravity;     /* m/s^2, acts along -z */
  double k_omega;     /* body-rate loop gain, 1/s */
  double drag[3];     /* diagonal of D (Eq. 2) */
  double u_min[5];    /* thrust N, rate cmd rad/s x3, progress accel */
  double u_max[5];
  double omega_max;   /* body-rate bound used by the feasibility penalty */
  double z_floor;     /* lowest altitude allowed by the penalty */
  /* input parameterisation: 0 collective thrust + body-rate command (CTBR),
   * 1 rotor-thrust rates u = dT/dt (Eq. 2 as printed) with the torque map
   * tau = (l/sqrt2 (T1+T2-T3-T4), l/sqrt2 (-T1+T2+T3-T4), c_tau (T1-T2+T3-T4)) */
  int32_t kind;
  double arm;         /* l, m */
  double c_tau;       /* rotor drag-torque coefficient, m */
  double thrust_min, thrust_max; /* rotor thrust range, N (the thrust saturates) */
} or_model;

typedef struct {
  int32_t objective;  /* 0 gate progress, 1 contouring, 2 tracking */
  int32_t K, N;
  double dt, lambda;
  double sigma[5];
  uint32_t seed, drone_id;
  double w_limit;      /* feasibility penalty weight */
  /* gate progress (Eq. 7) */
  double q_near, r_near;
  int32_t temporal_rule; /* 0 off, 1 time aligned, 2 same index */
  /* contouring (Eq. 9) */
  double q_lag, q_cont, q_omega[3], r_dv, r_dthrust, mu, v_theta_max;
  double theta_back, theta_ahead; /* projection window around last theta */
  /* tracking (Eq. 8) */
  double Q[13], QN[13], R[4];
  /* near-plane / near-edge reporting band, metres */
  double flag_eps;
  /* variants of the sampling and the warm start (Sec. III-B):
   * nominal_sample 1: sample 0 carries no perturbation (U^0 = U*, clamped);
   * warm_start 0: shift the new nominal by one step and repeat the last row,
   *            1: keep the complete new sequence as the next nominal */
  int32_t nominal_sample;
  int32_t warm_start;
} or_params;

typedef struct {
  int32_t n_gates, closed;
  const double* gates; /* [n][6] centre x y z, yaw, half width, half height */
  int32_t S;
  double L;            /* path length; nodes are L/S apart */
  const double* path;  /* [S][6] position, unit tangent */
  int32_t T;
  double dt_ref;       /* reference sample spacing, periodic in T*dt_ref */
  const double* ref;   /* [T][13] p v q w */
} or_track;

typedef struct {
  double* U;          /* [cap][5] nominal sequence, updated in place */
  int32_t n_nom;      /* valid rows in U (0: start from hover) */
  int32_t cap;        /* rows allocated in U and prevcnt */
  uint32_t iter;      /* Philox iteration counter */
  int32_t gate;       /* absolute index of the gate currently targeted */
  int32_t* prevcnt;   /* [cap] gates the previous nominal had passed by step k */
  int32_t n_prev;     /* valid entries in prevcnt (0: none yet) */
  double prev_x0[13];
  int32_t has_prev;
  double theta, v_theta, c_last;
  int32_t has_theta;
  double rotor[4];    /* rotor thrusts at x0 (rotor model): the controller's own */
  int32_t has_rotor;  /* integrated commands; hover thrust until set */
} or_state;

typedef struct {
  const double* Z_in; /* optional [N][K][5] normals to use instead of Philox */
  double* Z;          /* [N][K][5] normals used */
  double* J;          /* [K] cost */
  double* Jabs;       /* [K] sum of |stage terms| (relative-error scale) */
  int32_t* npass;     /* [K] gates passed inside the horizon */
  int32_t* first_pass;/* [K] step of the first accepted pass, -1 if none */
  int32_t* near_flag; /* [K] bit0 plane, bit1 edge, bit2 near-sphere */
  double* w;          /* [K] weights (Eq. 4) */
  double* Unew;       /* [N][5] weighted average before the shift (Eq. 5) */
  double* u0;         /* [5] */
  int32_t* passcnt;   /* [N+1] gates passed by state j of the new nominal */
  double* theta0;     /* [2] theta and v_theta at the start of this solve */
  double* xref;       /* [N+1][13] tracking reference window */
  double* Xnom;       /* [N+1][13] rollout of the new nominal */
  int32_t gate_at_start; /* gate index after the plant-crossing check */
  int32_t status;     /* 0 ok, 1 every cost non-finite (nominal kept) */
  double* Us;         /* [K][N][5] the clamped sampled sequences U^m (Eq. 3) */
} or_out;

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 Philox S-box with the */
/* two multipliers and the Weyl key schedule given there.                  */
/* ---------------------------------------------------------------------- */

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = M0 * (uint64_t)c0;
    uint64_t p1 = M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24 random bits to a uniform in (0, 1]; exact in binary32 and binary64. */
double or_uniform(uint32_t x) { return ((double)(x >> 8) + 1.0) * (1.0 / 16777216.0); }

/* Box-Muller: a pair of uniforms to a pair of independent standard normals. */
void or_box_muller(uint32_t xa, uint32_t xb, double z[2]) {
  const double two_pi = 6.283185307179586476925286766559;
  double ua = or_uniform(xa), ub = or_uniform(xb);
  double r = sqrt(-2.0 * log(ua));
  z[0] = r * cos(two_pi * ub);
  z[1] = r * sin(two_pi * ub);
}

/* Four standard normals for (sample m, step k, iteration, block). Eq. 3. */
void or_normals4(uint32_t seed, uint32_t drone, uint32_t m, uint32_t k,
                 uint32_t iter, uint32_t blk, double z[4]) {
  uint32_t ctr[4] = {m, k, iter, blk}, key[2] = {seed, drone}, x[4];
  or_philox4x32_10(ctr, key, x);
  or_box_muller(x[0], x[1], z);
  or_box_muller(x[2], x[3], z + 2);
}

/* ---------------------------------------------------------------------- */
/* Quadrotor model, Eq. 2, with the CTBR input                             */
/* x = [p(3) v(3) q(4: w x y z) omega(3)], u = [c, w_cmd(3)]               */
/* ---------------------------------------------------------------------- */

static void quat_to_R(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Eq. 2 for a collective thrust c along body z and a body torque tau */
static void rigid_deriv(const or_model* md, const double x[13], double c, const double tau[3], double dx[13]) {
  const double* v = x + 3; const double* q = x + 6; const double* w = x + 10;
  double R[9];
  quat_to_R(q, R);
  /* p_dot = v */
  dx[0] = v[0]; dx[1] = v[1]; dx[2] = v[2];
  /* v_dot = g + R T / m - R D R^T v, with T = (0, 0, c) */
  double Rtv[3], DRtv[3];
  for (int i = 0; i < 3; ++i) Rtv[i] = R[0 * 3 + i] * v[0] + R[1 * 3 + i] * v[1] + R[2 * 3 + i] * v[2];
  for (int i = 0; i < 3; ++i) DRtv[i] = md->drag[i] * Rtv[i];
  for (int i = 0; i < 3; ++i) {
    double thrust = R[i * 3 + 2] * c / md->mass;
    double drag = R[i * 3 + 0] * DRtv[0] + R[i * 3 + 1] * DRtv[1] + R[i * 3 + 2] * DRtv[2];
    dx[3 + i] = thrust - drag;
  }
  dx[5] -= md->gravity;
  /* q_dot = 1/2 Lambda(q) [0; omega]  (Hamilton product q * (0, omega)) */
  dx[6] = 0.5 * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
  dx[7] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
  dx[8] = 0.5 * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
  dx[9] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
  /* omega_dot = J^-1 (tau - omega x J omega) */
  const double* Jd = md->inertia;
  double Jw[3] = {Jd[0] * w[0], Jd[1] * w[1], Jd[2] * w[2]};
  double cx[3] = {w[1] * Jw[2] - w[2] * Jw[1], w[2] * Jw[0] - w[0] * Jw[2], w[0] * Jw[1] - w[1] * Jw[0]};
  for (int i = 0; i < 3; ++i) dx[10 + i] = (tau[i] - cx[i]) / Jd[i];
}

/* CTBR: u = (c, w_cmd), body-rate loop tau = J k_w (w_cmd - omega) */
void or_deriv(const or_model* md, const double x[13], const double u[4], double dx[13]) {
  const double* w = x + 10;
  double tau[3];
  for (int i = 0; i < 3; ++i) tau[i] = md->inertia[i] * md->k_omega * (u[1 + i] - w[i]);
  rigid_deriv(md, x, u[0], tau, dx);
}

/* Rotor model: collective thrust sum T_s and the torque map of Eq. 2 */
void or_deriv_rotor(const or_model* md, const double x[13], const double T[4], double dx[13]) {
  const double a = md->arm / sqrt(2.0);
  const double tau[3] = {a * (T[0] + T[1] - T[2] - T[3]), a * (-T[0] + T[1] + T[2] - T[3]),
                         md->c_tau * (T[0] - T[1] + T[2] - T[3])};
  rigid_deriv(md, x, T[0] + T[1] + T[2] + T[3], tau, dx);
}

/* Rotor thrusts a time t after T0 at the rates u (dT/dt = u held over the
 * step), saturating in [thrust_min, thrust_max]: the exact solution. */
void or_rotor_at(const or_model* md, const double T0[4], const double u[4], double t, double T[4]) {
  for (int s = 0; s < 4; ++s) {
    double v = T0[s] + u[s] * t;
    T[s] = v < md->thrust_min ? md->thrust_min : (v > md->thrust_max ? md->thrust_max : v);
  }
}

/* One classical Runge-Kutta step with the input held over the step. */
void or_rk4_step(const or_model* md, const double x[13], const double u[4], double h,
                 int renormalise, double xn[13]) {
  double k1[13], k2[13], k3[13], k4[13], xs[13];
  or_deriv(md, x, u, k1);
  for (int i = 0; i < 13; ++i) xs[i] = x[i] + 0.5 * h * k1[i];
  or_deriv(md, xs, u, k2);
  for (int i = 0; i < 13; ++i) xs[i] = x[i] + 0.5 * h * k2[i];
  or_deriv(md, xs, u, k3);
  for (int i = 0; i < 13; ++i) xs[i] = x[i] + h * k3[i];
  or_deriv(md, xs, u, k4);
  for (int i = 0; i < 13; ++i) xn[i] = x[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  if (renormalise) {
    double n = sqrt(xn[6] * xn[6] + xn[7] * xn[7] + xn[8] * xn[8] + xn[9] * xn[9]);
    for (int i = 6; i < 10; ++i) xn[i] /= n;
  }
}

/* One RK4 step of the rigid body with the rotor model: the stage thrusts
 * are the exact rotor thrusts at the stage times (T is not integrated). */
void or_rk4_step_rotor(const or_model* md, const double x[13], const double T0[4], const double u[4], double h,
                       int renormalise, double xn[13], double Tn[4]) {
  double k1[13], k2[13], k3[13], k4[13], xs[13], Th[4], T1[4];
  or_rotor_at(md, T0, u, 0.5 * h, Th);
  or_rotor_at(md, T0, u, h, T1);
  or_deriv_rotor(md, x, T0, k1);
  for (int i = 0; i < 13; ++i) xs[i] = x[i] + 0.5 * h * k1[i];
  or_deriv_rotor(md, xs, Th, k2);
  for (int i = 0; i < 13; ++i) xs[i] = x[i] + 0.5 * h * k2[i];
  or_deriv_rotor(md, xs, Th, k3);
  for (int i = 0; i < 13; ++i) xs[i] = x[i] + h * k3[i];
  or_deriv_rotor(md, xs, T1, k4);
  for (int i = 0; i < 13; ++i) xn[i] = x[i] + (h / 6.0) * (k1[i] + 2.0 * (k2[i] + k3[i]) + k4[i]);
  if (renormalise) {
    double n = sqrt(xn[6] * xn[6] + xn[7] * xn[7] + xn[8] * xn[8] + xn[9] * xn[9]);
    for (int i = 6; i < 10; ++i) xn[i] /= n;
  }
  for (int s = 0; s < 4; ++s) Tn[s] = T1[s];
}

/* Feasibility penalty ("external cost", Sec. III-B) on one state. */
double or_penalty(const or_model* md, const or_params* pr, const double x[13]) {
  double s = 0.0;
  for (int i = 0; i < 3; ++i) {
    double e = fabs(x[10 + i]) - md->omega_max;
    if (e > 0) s += e * e;
  }
  double zf = md->z_floor - x[2];
  if (zf > 0) s += zf * zf;
  return pr->w_limit * s;
}

/* ---------------------------------------------------------------------- */
/* Gates (Sec. IV-A)                                                        */
/* ---------------------------------------------------------------------- */

static const double* gate_row(const or_track* tr, int32_t idx) {
  int32_t n = tr->n_gates;
  int32_t i = tr->closed ? ((idx % n) + n) % n : (idx < n ? idx : n - 1);
  return tr->gates + 6 * i;
}

/* A pass is a crossing of the gate plane from its front (s < 0) to its back
 * (s >= 0) along the segment pa -> pb, through the opening: the crossing
 * point is within half_w laterally and half_h vertically of the centre.
 * Writes the signed distances and the opening offsets for the report band. */
int or_gate_crossing(const double g[6], const double pa[3], const double pb[3],
                     double info[4]) {
  double n[3] = {cos(g[3]), sin(g[3]), 0.0};
  double l[3] = {-sin(g[3]), cos(g[3]), 0.0};
  double sa = n[0] * (pa[0] - g[0]) + n[1] * (pa[1] - g[1]) + n[2] * (pa[2] - g[2]);
  double sb = n[0] * (pb[0] - g[0]) + n[1] * (pb[1] - g[1]) + n[2] * (pb[2] - g[2]);
  info[0] = sa; info[1] = sb; info[2] = 0.0; info[3] = 0.0;
  if (!(sa < 0.0 && sb >= 0.0)) return 0;
  double a = sa / (sa - sb);
  double e[3];
  for (int i = 0; i < 3; ++i) e[i] = pa[i] + a * (pb[i] - pa[i]) - g[i];
  double lat = l[0] * e[0] + l[1] * e[1] + l[2] * e[2];
  double vert = e[2];
  info[2] = lat; info[3] = vert;
  return fabs(lat) <= g[4] && fabs(vert) <= g[5];
}

/* ---------------------------------------------------------------------- */
/* Path and reference lookups (inputs of Algorithm 1)                       */
/* ---------------------------------------------------------------------- */

/* P_arc(theta): linear interpolation between uniform arc-length nodes of a
 * closed path; the tangent is interpolated the same way and renormalised. */
void or_path_eval(const or_track* tr, double theta, double P[3], double Tn[3]) {
  double ds = tr->L / tr->S;
  double th = fmod(theta, tr->L);
  if (th < 0) th += tr->L;
  double s = th / ds;
  int32_t j = (int32_t)floor(s);
  double f = s - j;
  if (j >= tr->S) { j = tr->S - 1; f = 1.0; }
  int32_t j1 = (j + 1) % tr->S;
  const double* a = tr->path + 6 * j; const double* b = tr->path + 6 * j1;
  for (int i = 0; i < 3; ++i) {
    P[i] = (1 - f) * a[i] + f * b[i];
    Tn[i] = (1 - f) * a[3 + i] + f * b[3 + i];
  }
  double n = sqrt(Tn[0] * Tn[0] + Tn[1] * Tn[1] + Tn[2] * Tn[2]);
  for (int i = 0; i < 3; ++i) Tn[i] /= n;
}

/* Arc length of the point of the path closest to p over the node segments
 * j in [jlo, jhi] (indices taken modulo S; the first minimum wins). */
double or_path_project(const or_track* tr, const double p[3], int32_t jlo, int32_t jhi) {
  double ds = tr->L / tr->S;
  double best = INFINITY, best_theta = 0.0;
  for (int32_t jj = jlo; jj <= jhi; ++jj) {
    int32_t j = ((jj % tr->S) + tr->S) % tr->S;
    int32_t j1 = (j + 1) % tr->S;
    const double* a = tr->path + 6 * j; const double* b = tr->path + 6 * j1;
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double r[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double t = (r[0] * d[0] + r[1] * d[1] + r[2] * d[2]) / dd;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    double e[3] = {r[0] - t * d[0], r[1] - t * d[1], r[2] - t * d[2]};
    double dist = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    if (dist < best) { best = dist; best_theta = (j + t) * ds; }
  }
  return best_theta;
}

/* x_ref(t) of the time-parameterised reference (periodic): linear in p, v,
 * omega; normalised linear blend of q on the shorter arc. */
void or_ref_eval(const or_track* tr, double t, double xr[13]) {
  double period = tr->T * tr->dt_ref;
  double tau = fmod(t, period);
  if (tau < 0) tau += period;
  double s = tau / tr->dt_ref;
  int32_t i = (int32_t)floor(s);
  double f = s - i;
  if (i >= tr->T) { i = tr->T - 1; f = 1.0; }
  int32_t i1 = (i + 1) % tr->T;
  const double* a = tr->ref + 13 * i; const double* b = tr->ref + 13 * i1;
  for (int c = 0; c < 13; ++c) xr[c] = (1 - f) * a[c] + f * b[c];
  double dot = a[6] * b[6] + a[7] * b[7] + a[8] * b[8] + a[9] * b[9];
  double sg = dot < 0 ? -1.0 : 1.0;
  double n2 = 0.0;
  for (int c = 6; c < 10; ++c) { xr[c] = (1 - f) * a[c] + f * sg * b[c]; n2 += xr[c] * xr[c]; }
  double n = sqrt(n2);
  for (int c = 6; c < 10; ++c) xr[c] /= n;
}

/* ---------------------------------------------------------------------- */
/* Stage costs                                                              */
/* ---------------------------------------------------------------------- */

static double dist2(const double a[3], const double b[3]) {
  double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
  return d0 * d0 + d1 * d1 + d2 * d2;
}

/* ||x - x_ref||^2_W with the quaternion error taken on the same hemisphere. */
static double track_err(const double x[13], const double xr[13], const double W[13]) {
  double s = 0.0;
  double dot = x[6] * xr[6] + x[7] * xr[7] + x[8] * xr[8] + x[9] * xr[9];
  double sg = dot < 0 ? -1.0 : 1.0;
  for (int c = 0; c < 13; ++c) {
    double r = (c >= 6 && c < 10) ? sg * xr[c] : xr[c];
    double e = x[c] - r;
    s += W[c] * e * e;
  }
  return s;
}

/* ---------------------------------------------------------------------- */
/* One solve (Algorithm 1, one iteration of the while loop)                 */
/* ---------------------------------------------------------------------- */

typedef struct {
  int32_t gate0;         /* absolute gate index at the start of the horizon */
  const int32_t* prev;   /* prevcnt, aligned to this solve's steps */
  int32_t n_prev;
  double theta0, vth0, c_last;
  const double* xref;    /* [N+1][13] */
} or_ctx;

static int32_t prev_at(const or_ctx* cx, int32_t k) {
  if (cx->n_prev <= 0) return 0;
  if (k < cx->n_prev) return cx->prev[k];
  return cx->prev[cx->n_prev - 1];
}

/* Rolls out one control sequence U[N][5] from x0 (and, for the rotor model,
 * the rotor thrusts T0) and scores it.  Returns J; fills the optional
 * diagnostics.  X (optional) receives [N+1][13], Trot [N+1][4]. */
static double rollout_cost(const or_model* md, const or_params* pr, const or_track* tr,
                           const or_ctx* cx, const double x0[13], const double* T0, const double* U,
                           double* Jabs_out, int32_t* npass_out, int32_t* first_out,
                           int32_t* flag_out, int32_t* passcnt_out, double* X, double* Trot) {
  int32_t N = pr->N;
  double x[13], xn[13];
  const int rotor = md->kind == 1;
  double Tk[4] = {0.0, 0.0, 0.0, 0.0}, Tk1[4] = {0.0, 0.0, 0.0, 0.0};  /* rotor thrusts at steps k, k+1 */
  if (rotor) memcpy(Tk, T0, sizeof Tk);
  if (Trot) memcpy(Trot, Tk, sizeof Tk);
  memcpy(x, x0, sizeof x);
  if (X) memcpy(X, x0, sizeof x);
  double J = 0.0, Jabs = 0.0;
  int32_t passed = 0, first = -1, flag = 0;
  int32_t gi = cx->gate0;
  const double* g0 = gate_row(tr, cx->gate0);
  double theta = cx->theta0, vth = cx->vth0, c_prev = cx->c_last;
  double eps = pr->flag_eps;
  if (passcnt_out) passcnt_out[0] = 0;
  for (int32_t k = 0; k < N; ++k) {
    const double* u = U + OR_NU * k;
    if (rotor)
      or_rk4_step_rotor(md, x, Tk, u, pr->dt, 1, xn, Tk1);
    else
      or_rk4_step(md, x, u, pr->dt, 1, xn);
    double pen = or_penalty(md, pr, xn);
    double stage = 0.0;
    if (pr->objective == 0) {
      /* Eq. 7: progress toward the gate targeted at the start of step k,
       * plus the conditional near-gate term on p_k and the current gate. */
      const double* g = gate_row(tr, gi);
      double prog = dist2(xn, g) - dist2(x, g);
      double d0 = sqrt(dist2(x, g0));
      double near = d0 < pr->r_near ? pr->q_near * d0 * d0 : 0.0;
      if (fabs(d0 - pr->r_near) < eps) flag |= 4;
      stage = prog + near;
      Jabs += fabs(dist2(xn, g)) + fabs(dist2(x, g)) + fabs(near);
      /* gate switching with the temporal-consistency rule (Sec. IV-A) */
      int last_gate = !tr->closed && gi >= tr->n_gates;
      double info[4];
      int cross = or_gate_crossing(g, x, xn, info);
      if (fabs(info[0]) < eps || fabs(info[1]) < eps) flag |= 1;
      if (info[0] < 0.0 && info[1] >= 0.0) {
        if (fabs(fabs(info[2]) - g[4]) < eps || fabs(fabs(info[3]) - g[5]) < eps) flag |= 2;
      }
      int ok_time = pr->temporal_rule == 0 || prev_at(cx, k) <= passed;
      if (cross && ok_time && !last_gate) {
        passed += 1;
        gi += 1;
        if (first < 0) first = k;
      }
    } else if (pr->objective == 1) {
      /* Eq. 9 with the progress state: v' = clamp(v + a dt), theta' by the
       * trapezoid; state terms on x_{k+1}. */
      double a = u[4];
      double v1 = vth + a * pr->dt;
      if (v1 < 0) v1 = 0;
      if (v1 > pr->v_theta_max) v1 = pr->v_theta_max;
      double th1 = theta + 0.5 * (vth + v1) * pr->dt;
      double P[3], Tn[3];
      or_path_eval(tr, th1, P, Tn);
      double e[3] = {xn[0] - P[0], xn[1] - P[1], xn[2] - P[2]};
      double et = e[0] * Tn[0] + e[1] * Tn[1] + e[2] * Tn[2];
      double el[3] = {et * Tn[0], et * Tn[1], et * Tn[2]};
      double ec[3] = {e[0] - el[0], e[1] - el[1], e[2] - el[2]};
      double lag = pr->q_lag * (el[0] * el[0] + el[1] * el[1] + el[2] * el[2]);
      double con = pr->q_cont * (ec[0] * ec[0] + ec[1] * ec[1] + ec[2] * ec[2]);
      double om = pr->q_omega[0] * xn[10] * xn[10] + pr->q_omega[1] * xn[11] * xn[11] +
                  pr->q_omega[2] * xn[12] * xn[12];
      double dv = pr->r_dv * a * a;
      /* thrust change: collective command (CTBR) or the rotor thrusts */
      double dT;
      if (rotor) {
        dT = 0.0;
        for (int s = 0; s < 4; ++s) dT += (Tk1[s] - Tk[s]) * (Tk1[s] - Tk[s]);
        dT *= pr->r_dthrust;
      } else {
        dT = pr->r_dthrust * (u[0] - c_prev) * (u[0] - c_prev);
      }
      double prog = pr->mu * v1;
      stage = lag + con + om + dv + dT - prog;
      Jabs += lag + con + om + dv + dT + fabs(prog);
      c_prev = u[0]; theta = th1; vth = v1;
    } else {
      /* Eq. 8: stage error on x_k (k < N), input effort about hover,
       * terminal error on x_N with Q_N. */
      const double* xr = cx->xref + 13 * k;
      double es = track_err(x, xr, pr->Q);
      /* input effort: about hover (CTBR), the thrust rates themselves (rotor) */
      double hover = rotor ? 0.0 : md->mass * md->gravity;
      double du[4] = {u[0] - hover, u[1], u[2], u[3]};
      double eu = pr->R[0] * du[0] * du[0] + pr->R[1] * du[1] * du[1] + pr->R[2] * du[2] * du[2] +
                  pr->R[3] * du[3] * du[3];
      stage = es + eu;
      if (k == N - 1) stage += track_err(xn, cx->xref + 13 * N, pr->QN);
      Jabs += stage;
    }
    J += stage + pen;
    Jabs += pen;
    memcpy(x, xn, sizeof x);
    if (rotor) memcpy(Tk, Tk1, sizeof Tk);
    if (X) memcpy(X + 13 * (k + 1), x, sizeof x);
    if (Trot) memcpy(Trot + 4 * (k + 1), Tk, sizeof Tk);
    if (passcnt_out) passcnt_out[k + 1] = passed;
  }
  if (Jabs_out) *Jabs_out = Jabs;
  if (npass_out) *npass_out = passed;
  if (first_out) *first_out = first;
  if (flag_out) *flag_out = flag;
  return J;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Geometric plant pass of the current gate between two consecutive solves. */
static int plant_passed(const or_track* tr, const or_state* st, const double x0[13]) {
  if (!st->has_prev) return 0;
  if (!tr->closed && st->gate >= tr->n_gates) return 0;
  double info[4];
  return or_gate_crossing(gate_row(tr, st->gate), st->prev_x0, x0, info);
}

int or_solve(const or_model* md, const or_params* pr, const or_track* tr, or_state* st,
             const double x0[13], double t0, or_out* out) {
  int32_t K = pr->K, N = pr->N;
  int32_t nu = pr->objective == 1 ? 5 : 4;
  double hover = md->mass * md->gravity;
  if (N > st->cap || K <= 0 || N <= 0) return -1;

  /* plant crossing since the last solve advances the gate (Sec. IV-A) */
  if (pr->objective == 0 && plant_passed(tr, st, x0)) {
    st->gate += 1;
    for (int32_t k = 0; k < st->n_prev; ++k) st->prevcnt[k] = st->prevcnt[k] > 0 ? st->prevcnt[k] - 1 : 0;
  }
  if (out) out->gate_at_start = st->gate;

  /* nominal sequence U* (Algorithm 1 initialises it; hover for CTBR) */
  double* Unom = (double*)malloc(sizeof(double) * OR_NU * N);
  for (int32_t k = 0; k < N; ++k) {
    for (int j = 0; j < OR_NU; ++j) {
      double v;
      if (st->n_nom > 0) v = st->U[OR_NU * (k < st->n_nom ? k : st->n_nom - 1) + j];
      else v = (j == 0 && md->kind != 1) ? hover : 0.0;  /* hover thrust (CTBR), zero rates (rotor) */
      Unom[OR_NU * k + j] = v;
    }
  }

  /* rotor thrusts at x0 (rotor model): the controller's integrated commands */
  double T0[4];
  for (int s = 0; s < 4; ++s) T0[s] = st->has_rotor ? st->rotor[s] : 0.25 * hover;

  or_ctx cx;
  memset(&cx, 0, sizeof cx);
  cx.gate0 = st->gate;
  cx.prev = st->prevcnt;
  cx.n_prev = st->n_prev;
  cx.c_last = st->has_prev ? st->c_last : hover;
  double* xref = NULL;
  if (pr->objective == 1) {
    double ds = tr->L / tr->S;
    int32_t jlo = 0, jhi = tr->S - 1;
    if (st->has_theta) {
      jlo = (int32_t)floor((st->theta - pr->theta_back) / ds);
      jhi = (int32_t)floor((st->theta + pr->theta_ahead) / ds);
    }
    cx.theta0 = or_path_project(tr, x0, jlo, jhi);
    cx.vth0 = st->has_theta ? st->v_theta : 0.0;
    if (out && out->theta0) { out->theta0[0] = cx.theta0; out->theta0[1] = cx.vth0; }
  } else if (pr->objective == 2) {
    xref = (double*)malloc(sizeof(double) * 13 * (N + 1));
    for (int32_t k = 0; k <= N; ++k) or_ref_eval(tr, t0 + k * pr->dt, xref + 13 * k);
    cx.xref = xref;
    if (out && out->xref) memcpy(out->xref, xref, sizeof(double) * 13 * (N + 1));
  }

  /* Eq. 3: sampled sequences, clamped to the input box */
  double* Us = (double*)malloc(sizeof(double) * (size_t)OR_NU * N * K);
  double* J = (double*)malloc(sizeof(double) * K);
  /* the samples are independent: a build with OpenMP (the timing baseline
   * on all host cores) runs them in parallel; the plain build ignores this */
#pragma omp parallel for schedule(dynamic, 16)
  for (int32_t m = 0; m < K; ++m) {
    for (int32_t k = 0; k < N; ++k) {
      double z[5] = {0, 0, 0, 0, 0};
      if (pr->nominal_sample && m == 0) {
        /* the unperturbed nominal is one of the candidates */
      } else if (out && out->Z_in) {
        for (int j = 0; j < OR_NU; ++j) z[j] = out->Z_in[((size_t)k * K + m) * OR_NU + j];
      } else {
        double z4[4];
        or_normals4(pr->seed, pr->drone_id, (uint32_t)m, (uint32_t)k, st->iter, 0u, z4);
        for (int j = 0; j < 4; ++j) z[j] = z4[j];
        if (nu == 5) {
          /* one block-1 draw serves four consecutive steps */
          or_normals4(pr->seed, pr->drone_id, (uint32_t)m, (uint32_t)(k & ~3), st->iter, 1u, z4);
          z[4] = z4[k & 3];
        }
      }
      if (out && out->Z)
        for (int j = 0; j < OR_NU; ++j) out->Z[((size_t)k * K + m) * OR_NU + j] = z[j];
      double* u = Us + ((size_t)m * N + k) * OR_NU;
      for (int j = 0; j < OR_NU; ++j) {
        if (j < nu) u[j] = clampd(Unom[OR_NU * k + j] + pr->sigma[j] * z[j], md->u_min[j], md->u_max[j]);
        else u[j] = 0.0;
      }
    }
    if (out && out->Us) memcpy(out->Us + (size_t)m * N * OR_NU, Us + (size_t)m * N * OR_NU, sizeof(double) * OR_NU * N);
    /* rollout and objective for this sample (Algorithm 1 inner loop) */
    double jabs;
    int32_t np, fp, fl;
    J[m] = rollout_cost(md, pr, tr, &cx, x0, T0, Us + (size_t)m * N * OR_NU, &jabs, &np, &fp, &fl, NULL, NULL,
                        NULL);
    if (out && out->J) out->J[m] = J[m];
    if (out && out->Jabs) out->Jabs[m] = jabs;
    if (out && out->npass) out->npass[m] = np;
    if (out && out->first_pass) out->first_pass[m] = fp;
    if (out && out->near_flag) out->near_flag[m] = fl;
  }

  /* Eq. 4: w_m = exp(-J_m / lambda) / sum_i exp(-J_i / lambda), evaluated
   * with the minimum cost factored out of numerator and denominator. */
  double Jmin = INFINITY;
  for (int32_t m = 0; m < K; ++m) if (isfinite(J[m]) && J[m] < Jmin) Jmin = J[m];
  double* w = (double*)malloc(sizeof(double) * K);
  int status = 0;
  double* Unew = (double*)malloc(sizeof(double) * OR_NU * N);
  if (!isfinite(Jmin)) {
    status = 1;
    for (int32_t m = 0; m < K; ++m) w[m] = 0.0;
    memcpy(Unew, Unom, sizeof(double) * OR_NU * N);
  } else {
    double S = 0.0;
    for (int32_t m = 0; m < K; ++m) {
      w[m] = isfinite(J[m]) ? exp(-(J[m] - Jmin) / pr->lambda) : 0.0;
      S += w[m];
    }
    for (int32_t m = 0; m < K; ++m) w[m] /= S;
    /* Eq. 5: U* = sum_m w_m U^m */
    for (int32_t k = 0; k < N; ++k)
      for (int j = 0; j < OR_NU; ++j) {
        double s = 0.0;
        if (j < nu)
          for (int32_t m = 0; m < K; ++m) s += w[m] * Us[((size_t)m * N + k) * OR_NU + j];
        Unew[OR_NU * k + j] = s;
      }
  }
  if (out && out->w) memcpy(out->w, w, sizeof(double) * K);
  if (out && out->Unew) memcpy(out->Unew, Unew, sizeof(double) * OR_NU * N);
  if (out && out->u0) memcpy(out->u0, Unew, sizeof(double) * OR_NU);

  /* rollout of the new nominal: gate pass counts for the next solve's
   * temporal rule (and the predicted trajectory) */
  int32_t* pc = (int32_t*)malloc(sizeof(int32_t) * (N + 1));
  double* Xn = (double*)malloc(sizeof(double) * 13 * (N + 1));
  rollout_cost(md, pr, tr, &cx, x0, T0, Unew, NULL, NULL, NULL, NULL, pc, Xn, NULL);
  if (out && out->passcnt) memcpy(out->passcnt, pc, sizeof(int32_t) * (N + 1));
  if (out && out->Xnom) memcpy(out->Xnom, Xn, sizeof(double) * 13 * (N + 1));

  /* warm start (Sec. III-B): shift by one step and repeat the last row, or
   * keep the complete sequence */
  for (int32_t k = 0; k < N; ++k) {
    int32_t src = pr->warm_start == 1 ? k : (k + 1 < N ? k + 1 : N - 1);
    for (int j = 0; j < OR_NU; ++j) st->U[OR_NU * k + j] = Unew[OR_NU * src + j];
  }
  st->n_nom = N;
  /* pass counts seen from the next solve: time aligned = one step later */
  for (int32_t k = 0; k < N; ++k) {
    int32_t src = pr->temporal_rule == 2 ? k : k + 1;
    st->prevcnt[k] = pc[src];
  }
  st->n_prev = N;
  if (pr->objective == 1) {
    double v1 = clampd(cx.vth0 + Unew[4] * pr->dt, 0.0, pr->v_theta_max);
    st->theta = cx.theta0;
    st->v_theta = v1;
    st->has_theta = 1;
  }
  st->c_last = Unew[0];
  if (md->kind == 1) {
    /* the plant applies u0 (rotor-thrust rates) for one control period */
    or_rotor_at(md, T0, Unew, pr->dt, st->rotor);
    st->has_rotor = 1;
  }
  memcpy(st->prev_x0, x0, sizeof(double) * 13);
  st->has_prev = 1;
  st->iter += 1;
  if (out) out->status = status;

  free(Unom); free(xref); free(Us); free(J); free(w); free(Unew); free(pc); free(Xn);
  return status;
}

/* Threads the sample loop of or_solve uses (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int or_threads(void) { return omp_get_max_threads(); }
#else
int or_threads(void) { return 1; }
#endif

/* Plain rollout of a given sequence (no sampling), for the model tests. */
double or_rollout(const or_model* md, const or_params* pr, const or_track* tr, const double x0[13],
                  const double* U, int32_t gate0, const int32_t* prev, int32_t n_prev,
                  double theta0, double vth0, double c_last, const double* xref,
                  double* X, int32_t* passcnt, const double* T0, double* Trot) {
  or_ctx cx;
  memset(&cx, 0, sizeof cx);
  cx.gate0 = gate0; cx.prev = prev; cx.n_prev = n_prev;
  cx.theta0 = theta0; cx.vth0 = vth0; cx.c_last = c_last; cx.xref = xref;
  return rollout_cost(md, pr, tr, &cx, x0, T0, U, NULL, NULL, NULL, NULL, passcnt, X, Trot);
}
