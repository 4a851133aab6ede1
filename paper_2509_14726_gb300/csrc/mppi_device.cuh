// mppi_device.cuh -- device-side data layout and per-thread arithmetic of one
// MPPI solve (arXiv 2509.14726, Sec. III-IV) for sm_103a.
//
// One thread owns one sample: its 13-D state lives in registers for the whole
// horizon, positions and velocities carry a compensation term (Kahan), and the
// cost is accumulated in a float hi/lo pair.  Everything a block shares (the
// nominal U*, gates, path table, reference window) sits in shared memory.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/mppi.h"

namespace mppi {

constexpr int kNX = 13;
constexpr int kNU = 5;
constexpr int kMaxN = MPPI_MAX_N;
constexpr int kMaxGates = MPPI_MAX_GATES;
constexpr int kMaxBlock = 512;

// --------------------------------------------------------------------------
// resident per-drone controller state (device memory, one per handle)
// --------------------------------------------------------------------------
struct DevState {
  int32_t gate;        // absolute index of the targeted gate
  uint32_t iter;       // Philox iteration (counter word 2)
  int32_t has_prev;    // prev_x0 valid
  int32_t has_theta;   // theta / v_theta valid (contouring)
  int32_t n_nom;       // rows of U that came from a solve (0: hover init)
  int32_t n_prev;      // entries of prevcnt that came from a solve
  int32_t gate0;       // gate index at the start of the last solve
  int32_t adv;         // gates the plant passed between the last two solves
  int32_t status;      // mppi_status of the last solve
  int32_t timeouts;    // bounded waits that gave up (diagnostics)
  double theta;        // progress at the start of the last solve
  double v_theta;      // progress speed for the next solve
  float c_last;        // last applied collective thrust
  float prev_x0[kNX];  // x0 of the last solve
  double scal[4];      // theta0, v_theta0, J_min, sum of exp weights
  float rotor[4];      // rotor model: rotor thrusts at the next x0 (integrated commands)
  float rotor_prev[4]; // rotor thrusts at the x0 of the last solve (its nominal rollout)
  int32_t has_rotor;   // 0: hover thrust
  int32_t timeouts_seen;  // value of timeouts when the last solve ended
};

// Step constants as (hi, lo) binary32 pairs, so that the RK4 weights h/6,
// h^2/6, h/12 and the factor 1/m carry no systematic rounding bias (a bias
// of a constant factor integrates linearly over the horizon, where random
// rounding only random-walks):
//   c[0] = (h/6, lo, h^2/6, lo), c[1] = (h/12, lo, 1/m lo part, 0).
// Kept in shared memory and read where used.
struct StepConsts {
  float4 c[2];
};

// gate frame: centre, plane normal (horizontal), half sizes; a handle keeps
// one per gate in device memory, and the rollout stages them in shared
// memory by a bulk copy (32 bytes each, read as two float4)
struct __align__(16) GateF {
  float cx, cy, cz, nx, ny, hw, hh, pad;
};

// --------------------------------------------------------------------------
// per-handle solve descriptor (device memory, read by every block)
// --------------------------------------------------------------------------
struct SolveDesc {
  StepConsts stepc;     // RK4 weights and 1/m as (hi, lo) pairs (first: 16-byte aligned)
  // model (Eq. 2, CTBR input)
  float mass, inv_mass, gravity, k_omega;
  float gyro[3];        // (Jz-Jy)/Jx, (Jx-Jz)/Jy, (Jy-Jx)/Jz
  float drag[3];
  int32_t has_drag;
  float u_min[kNU], u_max[kNU];
  float omega_max, z_floor;
  // sampling and weights (Eq. 3, Eq. 4)
  int32_t objective, K, N, nu;
  float dt, lambda, inv_lambda;
  float sigma[kNU];
  uint32_t seed, drone_id;
  int32_t noise_bf16, accum;
  // costs
  float w_limit, q_near, r_near2;
  int32_t temporal_rule;
  float q_lag, q_cont, q_omega[3], r_dv, r_dthrust, mu, v_theta_max, theta_back, theta_ahead;
  float Q[kNX], QN[kNX], R[4];
  float hover;
  // track (device pointers)
  const float* gates;   // [n][6] centre, yaw, half width, half height
  const GateF* gframes; // [n] the frames of those gates (built once per handle)
  int32_t n_gates, closed;
  const float* path;    // [S][6]
  int32_t S;
  float L, ds, inv_ds;
  const float* ref;     // [T][13] (16-byte aligned)
  int32_t T;
  float dt_ref;
  int32_t ref_rows;     // reference rows a tracking block stages in shared memory (0: reads them from ref)
  int32_t ref_pad;      // bytes readable past the end of ref (a bulk copy is rounded up to 16 bytes)
  // resident state
  DevState* st;
  float* U;             // [N_cap][5] (+pad), always fully populated
  int32_t* prevcnt;     // [N_cap] (+pad), always fully populated
  int32_t N_cap;
  // per-solve buffers
  float4* Z4;           // [N][K] standard normals (F32 storage)
  uint2* Zb;            // [N][K] 4 x bf16 (BF16 storage)
  float* Z5;            // [N][K] 5th normal (contouring, F32)
  __nv_bfloat16* Z5b;   // [N][K] 5th normal (contouring, BF16)
  double* J;            // [K] cost as a (hi, lo) float pair per 8-byte slot: J = hi + lo
  int32_t* info;        // [K] npass | (first_pass + 1) << 16
  double* part_m;       // [tiles] per-tile minimum cost
  double* part_S;       // [tiles] per-tile sum of exp weights
  double* part_P;       // [tiles][N][5] per-tile weighted deviation sums
  uint32_t* ticket;     // blocks of this solve that finished
  float* unew;          // [N][5] Eq. 5 result before the shift
  int32_t* passcnt;     // [N+1] gates passed along the new nominal
  float* xref;          // [N+1][13] tracking window used (diagnostics)
  int32_t n_tiles, block;
  int32_t ext_noise;    // 1: use the caller's noise for this solve
  int32_t noise_gen;    // MPPI_NOISEGEN_*: where the normals are drawn
  int32_t nominal_sample;  // 1: sample 0 carries no perturbation
  int32_t warm_keep;    // 1: the next nominal is the whole new sequence (no shift)
  // rotor-thrust-rate model (model kind MPPI_MODEL_ROTOR_RATE)
  int32_t rotor;
  float arm2, c_tau, thrust_min, thrust_max, inv_J[3];
  float kt[3][2];       // torque factors l/sqrt2/Jx, l/sqrt2/Jy, c_tau/Jz as (hi, lo)
  int32_t spt;          // samples per thread: a tile holds block x spt samples
  uint32_t wait_ns;     // limit of the rollout's first wait for its bulk copies
  int32_t wait_unreachable;  // testing: that wait targets a barrier nothing completes
};

// samples one rollout block covers
__host__ __device__ inline int tile_samples(const SolveDesc& d) { return d.block * d.spt; }

// device-side per-launch inputs and outputs (indexed by the solve's position
// in the batch); pointers may be device or mapped host memory
struct LaunchIO {
  const float* x0;      // [n][13]; nullptr: use x0v (single solve)
  const double* t0;     // [n];     nullptr: use t0v
  float* u0;            // [n][5]
  int32_t* status;      // [n] mppi_status of each solve (may be nullptr)
  float x0v[kNX];
  double t0v;
};

// tile -> (solve position, first sample)
struct Tile {
  int32_t solve;
  int32_t m0;
};

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    // one 32x32 -> 64-bit product per multiplier gives both halves
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// uniform in (0, 1] from the top 24 bits; exact in binary32
__device__ __forceinline__ float u24(uint32_t x) { return (float)((x >> 8) + 1u) * 5.9604644775390625e-8f; }

__device__ __forceinline__ float2 box_muller(uint32_t xa, uint32_t xb) {
  const float r = sqrtf(-2.0f * logf(u24(xa)));
  float s, c;
  sincospif(2.0f * u24(xb), &s, &c);
  return make_float2(r * c, r * s);
}

__device__ __forceinline__ float4 normals4(uint32_t seed, uint32_t drone, uint32_t m, uint32_t k,
                                           uint32_t iter, uint32_t blk) {
  const uint4 x = philox4x32_10(make_uint4(m, k, iter, blk), seed, drone);
  const float2 a = box_muller(x.x, x.y), b = box_muller(x.z, x.w);
  return make_float4(a.x, a.y, b.x, b.y);
}

// The 5th (progress) normal of (sample m, step k), contouring: the four
// normals of block 1 at step 4 floor(k / 4) serve steps 4j .. 4j+3 in order,
// so this draws one Philox block and the one Box-Muller pair step k needs.
__device__ __forceinline__ float normal5(uint32_t seed, uint32_t drone, uint32_t m, uint32_t k, uint32_t iter) {
  const uint4 x = philox4x32_10(make_uint4(m, k & ~3u, iter, 1u), seed, drone);
  const bool hi = (k & 2u) != 0u;
  const float2 z = box_muller(hi ? x.z : x.x, hi ? x.w : x.y);
  return (k & 1u) ? z.y : z.x;
}

// --------------------------------------------------------------------------
// small helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// Kahan step: s + y with the running compensation c (true sum ~ s - c)
__device__ __forceinline__ void kahan_add(float& s, float& c, float y) {
  const float yy = y - c;
  const float t = s + yy;
  c = (t - s) - yy;
  s = t;
}

// error-free sum (Knuth TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// --------------------------------------------------------------------------
// quadrotor state and the RK4 step (Eq. 2 with CTBR; classical RK4, ZOH input)
// --------------------------------------------------------------------------
struct Quad {
  float px, py, pz, cpx, cpy, cpz;  // position + Kahan compensation
  float vx, vy, vz, cvx, cvy, cvz;  // velocity + Kahan compensation
  float qw, qx, qy, qz;             // attitude
  float cqw, cqx, cqy, cqz;         // its Kahan compensation (true q = q - cq)
  float wx, wy, wz;
  float cwx, cwy, cwz;              // body-rate compensation (rotor model only)
};

struct ModelRegs {
  float inv_mass, gravity, k_omega, g0, g1, g2, d0, d1, d2;
  int has_drag;
};

// |q|^2 - 1 for a quaternion whose norm is 1 up to binary32 rounding: exact
// products (FMA) and error-free sums, so that the result is accurate to
// about 1e-14 instead of one rounding of |q|^2 (6e-8).
__device__ __forceinline__ float quat_norm_excess(float w, float x, float y, float z) {
  float s = w * w;
  float e = fmaf(w, w, -s);
  const float v[3] = {x, y, z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float p = v[i] * v[i];
    const float pe = fmaf(v[i], v[i], -p);
    const float t = s + p;
    const float bb = t - s;
    e += ((s - (t - bb)) + (p - bb)) + pe;
    s = t;
  }
  return (s - 1.f) + e;
}

// A shared-memory vector load the compiler keeps where it is written (not
// hoisted out of a loop into registers).
__device__ __forceinline__ float4 lds4_volatile(const float4* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return v;
}

// a state from the 13 floats of x0
__device__ __forceinline__ void quad_init(Quad& s, const float* x0) {
  s.px = x0[0]; s.py = x0[1]; s.pz = x0[2];
  s.cpx = s.cpy = s.cpz = 0.f;
  s.vx = x0[3]; s.vy = x0[4]; s.vz = x0[5];
  s.cvx = s.cvy = s.cvz = 0.f;
  s.qw = x0[6]; s.qx = x0[7]; s.qy = x0[8]; s.qz = x0[9];
  s.cqw = s.cqx = s.cqy = s.cqz = 0.f;
  s.wx = x0[10]; s.wy = x0[11]; s.wz = x0[12];
  s.cwx = s.cwy = s.cwz = 0.f;
}

// c/m from the pair (inv_mass, lo): the correctly rounded product instead of
// c * round(1/m), whose bias is the same on every step
__device__ __forceinline__ float thrust_accel(float c, float inv_mass, float inv_mass_lo) {
  const float a = c * inv_mass;
  return a + fmaf(c, inv_mass_lo, fmaf(c, inv_mass, -a));
}

// The RK4 combination of the attitude: q <- (q + D) / |q + D| with
// D = h/12 (k1 + 2 k2 + 2 k3 + k4) of the doubled quaternion rate.  With
// |q|^2 = 1 + qe, delta = |q + D|^2 - 1 = qe + 2 q.D + |D|^2: both terms are
// small (D is nearly orthogonal to q), so delta is accurate in binary32, and
// 1/sqrt(1 + delta) - 1 = -delta/2 + 3 delta^2/8 - ...  The renormalised
// increment D + (q + D) e goes into the compensated q with one Kahan step per
// component; no component is rounded back to binary32.
// qe: |q|^2 - 1 before the step (quat_norm_excess of x0's quaternion on the
// first step; 0 afterwards, since every step leaves |q| = 1).
__device__ __forceinline__ void quat_advance(Quad& s, float qe, float Dw, float Dx, float Dy, float Dz) {
  const float qd = s.qw * Dw + s.qx * Dx + s.qy * Dy + s.qz * Dz;
  const float d2 = Dw * Dw + Dx * Dx + Dy * Dy + Dz * Dz;
  const float dd = qe + fmaf(2.f, qd, d2);
  const float e = fabsf(dd) < 1e-3f ? dd * fmaf(0.375f, dd, -0.5f) : rsqrtf(1.f + dd) - 1.f;
  kahan_add(s.qw, s.cqw, fmaf(s.qw + Dw, e, Dw));
  kahan_add(s.qx, s.cqx, fmaf(s.qx + Dx, e, Dx));
  kahan_add(s.qy, s.cqy, fmaf(s.qy + Dy, e, Dy));
  kahan_add(s.qz, s.cqz, fmaf(s.qz + Dz, e, Dz));
}

// v += (h/6) a with the constant as a pair: the increment's product error and
// the constant's low part go into the compensation
__device__ __forceinline__ void vel_advance(float& v, float& cv, float a, float h6, float h6l) {
  const float y = h6 * a;
  const float lo = fmaf(h6l, a, fmaf(h6, a, -y));
  kahan_add(v, cv, y);
  cv -= lo;
}

// Body-z thrust acceleration R(q) e_z c/m - g e_z, with the factor 2 of R
// folded into ac2 = 2 c/m and acg = c/m - g (both per step).
__device__ __forceinline__ void accel_nodrag(float ac2, float acg, float qw, float qx, float qy, float qz, float& ax,
                                             float& ay, float& az) {
  ax = ac2 * (qx * qz + qw * qy);
  ay = ac2 * (qy * qz - qw * qx);
  az = acg - ac2 * (qx * qx + qy * qy);
}

// the same plus the body-frame drag - R D R^T v
__device__ __forceinline__ void accel_drag(const ModelRegs& M, float ac2, float acg, float qw, float qx, float qy,
                                           float qz, float vx, float vy, float vz, float& ax, float& ay, float& az) {
  accel_nodrag(ac2, acg, qw, qx, qy, qz, ax, ay, az);
  const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz), r02 = 2.f * (qx * qz + qw * qy);
  const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz), r12 = 2.f * (qy * qz - qw * qx);
  const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx), r22 = 1.f - 2.f * (qx * qx + qy * qy);
  const float bv0 = M.d0 * (r00 * vx + r10 * vy + r20 * vz);
  const float bv1 = M.d1 * (r01 * vx + r11 * vy + r21 * vz);
  const float bv2 = M.d2 * (r02 * vx + r12 * vy + r22 * vz);
  ax -= r00 * bv0 + r01 * bv1 + r02 * bv2;
  ay -= r10 * bv0 + r11 * bv1 + r12 * bv2;
  az -= r20 * bv0 + r21 * bv1 + r22 * bv2;
}

// Twice the quaternion rate, q * (0, w) (the 1/2 of Eq. 2 is folded into the
// step sizes), and the body-rate derivative k_w (w_cmd - w) - J^-1 (w x J w)
// with kc = k_w w_cmd precomputed per step.
__device__ __forceinline__ void attitude_rate2(const ModelRegs& M, float kcx, float kcy, float kcz, float qw,
                                               float qx, float qy, float qz, float wx, float wy, float wz, float& dqw,
                                               float& dqx, float& dqy, float& dqz, float& dwx, float& dwy,
                                               float& dwz) {
  dqw = -(qx * wx + qy * wy + qz * wz);
  dqx = qw * wx + qy * wz - qz * wy;
  dqy = qw * wy + qz * wx - qx * wz;
  dqz = qw * wz + qx * wy - qy * wx;
  dwx = kcx - M.k_omega * wx - M.g0 * wy * wz;
  dwy = kcy - M.k_omega * wy - M.g1 * wz * wx;
  dwz = kcz - M.k_omega * wz - M.g2 * wx * wy;
}

// One classical RK4 step (Eq. 2 with the CTBR input held over the step).
// Writes the position increment (exact RK4 increment, before the compensated
// accumulation) to dp.  Without drag the accelerations depend on q only, so
// the stage velocities are not formed:  p += h v + h^2/6 (a1 + a2 + a3),
// v += h/6 (a1 + 2 a2 + 2 a3 + a4).
// sc: the solve's StepConsts in shared memory; qe: |q|^2 - 1 at the start of
// the step (see quat_advance).
template <bool DRAG>
__device__ __forceinline__ void rk4_step(const ModelRegs& M, const StepConsts* sc, Quad& s, float qe, float c,
                                         float cx, float cy, float cz, float h, float& dpx, float& dpy,
                                         float& dpz) {
  const float4 c1 = lds4_volatile(&sc->c[1]);
  const float ac = thrust_accel(c, M.inv_mass, c1.z);
  const float ac2 = 2.f * ac, acg = ac - M.gravity;
  const float kcx = M.k_omega * cx, kcy = M.k_omega * cy, kcz = M.k_omega * cz;
  const float h2 = 0.5f * h, h4 = 0.25f * h;
  float dqw, dqx, dqy, dqz, dwx, dwy, dwz, ax, ay, az;
  // stage 1
  attitude_rate2(M, kcx, kcy, kcz, s.qw, s.qx, s.qy, s.qz, s.wx, s.wy, s.wz, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, s.qw, s.qx, s.qy, s.qz, s.vx, s.vy, s.vz, ax, ay, az);
  else
    accel_nodrag(ac2, acg, s.qw, s.qx, s.qy, s.qz, ax, ay, az);
  float sqw = dqw, sqx = dqx, sqy = dqy, sqz = dqz, swx = dwx, swy = dwy, swz = dwz;
  float sax = ax, say = ay, saz = az;  // a1 + 2 a2 + 2 a3 + a4
  float pax = ax, pay = ay, paz = az;  // a1 + a2 + a3
  float vx2 = 0.f, vy2 = 0.f, vz2 = 0.f;
  // stage 2
  float qw2 = s.qw + h4 * dqw, qx2 = s.qx + h4 * dqx, qy2 = s.qy + h4 * dqy, qz2 = s.qz + h4 * dqz;
  float wx2 = s.wx + h2 * dwx, wy2 = s.wy + h2 * dwy, wz2 = s.wz + h2 * dwz;
  if (DRAG) { vx2 = s.vx + h2 * ax; vy2 = s.vy + h2 * ay; vz2 = s.vz + h2 * az; }
  attitude_rate2(M, kcx, kcy, kcz, qw2, qx2, qy2, qz2, wx2, wy2, wz2, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, qw2, qx2, qy2, qz2, vx2, vy2, vz2, ax, ay, az);
  else
    accel_nodrag(ac2, acg, qw2, qx2, qy2, qz2, ax, ay, az);
  sqw += 2.f * dqw; sqx += 2.f * dqx; sqy += 2.f * dqy; sqz += 2.f * dqz;
  swx += 2.f * dwx; swy += 2.f * dwy; swz += 2.f * dwz;
  sax += 2.f * ax; say += 2.f * ay; saz += 2.f * az;
  pax += ax; pay += ay; paz += az;
  // stage 3
  qw2 = s.qw + h4 * dqw; qx2 = s.qx + h4 * dqx; qy2 = s.qy + h4 * dqy; qz2 = s.qz + h4 * dqz;
  wx2 = s.wx + h2 * dwx; wy2 = s.wy + h2 * dwy; wz2 = s.wz + h2 * dwz;
  if (DRAG) { vx2 = s.vx + h2 * ax; vy2 = s.vy + h2 * ay; vz2 = s.vz + h2 * az; }
  attitude_rate2(M, kcx, kcy, kcz, qw2, qx2, qy2, qz2, wx2, wy2, wz2, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, qw2, qx2, qy2, qz2, vx2, vy2, vz2, ax, ay, az);
  else
    accel_nodrag(ac2, acg, qw2, qx2, qy2, qz2, ax, ay, az);
  sqw += 2.f * dqw; sqx += 2.f * dqx; sqy += 2.f * dqy; sqz += 2.f * dqz;
  swx += 2.f * dwx; swy += 2.f * dwy; swz += 2.f * dwz;
  sax += 2.f * ax; say += 2.f * ay; saz += 2.f * az;
  pax += ax; pay += ay; paz += az;
  // stage 4
  qw2 = s.qw + h2 * dqw; qx2 = s.qx + h2 * dqx; qy2 = s.qy + h2 * dqy; qz2 = s.qz + h2 * dqz;
  wx2 = s.wx + h * dwx; wy2 = s.wy + h * dwy; wz2 = s.wz + h * dwz;
  if (DRAG) { vx2 = s.vx + h * ax; vy2 = s.vy + h * ay; vz2 = s.vz + h * az; }
  attitude_rate2(M, kcx, kcy, kcz, qw2, qx2, qy2, qz2, wx2, wy2, wz2, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, qw2, qx2, qy2, qz2, vx2, vy2, vz2, ax, ay, az);
  else
    accel_nodrag(ac2, acg, qw2, qx2, qy2, qz2, ax, ay, az);
  sqw += dqw; sqx += dqx; sqy += dqy; sqz += dqz;
  swx += dwx; swy += dwy; swz += dwz;
  sax += ax; say += ay; saz += az;
  // combine: p and v compensated with the weights as (hi, lo) pairs, q
  // compensated and renormalised exactly (quat_advance), w plain (the rate
  // loop damps its rounding)
  const float4 c0 = lds4_volatile(&sc->c[0]);  // (h/6, lo, h^2/6, lo)
  dpx = h * s.vx + c0.z * pax;
  dpy = h * s.vy + c0.z * pay;
  dpz = h * s.vz + c0.z * paz;
  kahan_add(s.px, s.cpx, dpx);
  kahan_add(s.py, s.cpy, dpy);
  kahan_add(s.pz, s.cpz, dpz);
  s.cpx -= c0.w * pax;
  s.cpy -= c0.w * pay;
  s.cpz -= c0.w * paz;
  vel_advance(s.vx, s.cvx, sax, c0.x, c0.y);
  vel_advance(s.vy, s.cvy, say, c0.x, c0.y);
  vel_advance(s.vz, s.cvz, saz, c0.x, c0.y);
  s.wx += c0.x * swx;
  s.wy += c0.x * swy;
  s.wz += c0.x * swz;
  quat_advance(s, qe, fmaf(c1.y, sqw, c1.x * sqw), fmaf(c1.y, sqx, c1.x * sqx), fmaf(c1.y, sqy, c1.x * sqy),
               fmaf(c1.y, sqz, c1.x * sqz));
}

// Rotor-thrust-rate model (Eq. 2 as printed): four rotor thrusts with
// dT/dt = u held over the step, saturating in [tmin, tmax]; collective
// thrust = their sum; torque tau = (l/sqrt2 (T0+T1-T2-T3),
// l/sqrt2 (-T0+T1+T2-T3), c_tau (T0-T1+T2-T3)).
struct RotorRegs {
  float tmin, tmax;
  float kx, kxl, ky, kyl, kz, kzl;  // l/sqrt2/Jx, l/sqrt2/Jy, c_tau/Jz as (hi, lo) pairs
};

__host__ __device__ inline RotorRegs rotor_regs(const SolveDesc& d) {
  RotorRegs R;
  R.tmin = d.thrust_min;
  R.tmax = d.thrust_max;
  R.kx = d.kt[0][0]; R.kxl = d.kt[0][1];
  R.ky = d.kt[1][0]; R.kyl = d.kt[1][1];
  R.kz = d.kt[2][0]; R.kzl = d.kt[2][1];
  return R;
}

// k * x with the constant k as a (hi, lo) pair: the correctly rounded product
__device__ __forceinline__ float pair_mul(float k, float kl, float x) {
  const float a = k * x;
  return a + fmaf(kl, x, fmaf(k, x, -a));
}

// twice the quaternion rate and the body-rate derivative J^-1 tau - J^-1 (w x J w)
// for the torque accelerations (bx, by, bz) = J^-1 tau
__device__ __forceinline__ void attitude_rate2_torque(const ModelRegs& M, float bx, float by, float bz, float qw,
                                                      float qx, float qy, float qz, float wx, float wy, float wz,
                                                      float& dqw, float& dqx, float& dqy, float& dqz, float& dwx,
                                                      float& dwy, float& dwz) {
  dqw = -(qx * wx + qy * wy + qz * wz);
  dqx = qw * wx + qy * wz - qz * wy;
  dqy = qw * wy + qz * wx - qx * wz;
  dqz = qw * wz + qx * wy - qy * wx;
  dwx = bx - M.g0 * wy * wz;
  dwy = by - M.g1 * wz * wx;
  dwz = bz - M.g2 * wx * wy;
}

// thrust terms of one set of rotor thrusts: 2 c/m, c/m - g and J^-1 tau.
// The torque combinations are formed from pairwise differences of the
// (nearly equal) thrusts, which are exact when the two are within a factor
// of two, instead of differences of sums, which cancel.
__device__ __forceinline__ void rotor_forces(const ModelRegs& M, const RotorRegs& R, float iml, float t0, float t1,
                                             float t2, float t3, float& ac2, float& acg, float& bx, float& by,
                                             float& bz) {
  const float ac = thrust_accel((t0 + t1) + (t2 + t3), M.inv_mass, iml);
  ac2 = 2.f * ac;
  acg = ac - M.gravity;
  // the torque factors are constants: correctly rounded products, no bias
  bx = pair_mul(R.kx, R.kxl, (t0 - t2) + (t1 - t3));
  by = pair_mul(R.ky, R.kyl, (t1 - t0) + (t2 - t3));
  bz = pair_mul(R.kz, R.kzl, (t0 - t1) + (t2 - t3));
}

// One compensated step of a saturating thrust ramp: (T, c) holds T - c, the
// increment y is added with Kahan's correction; a bound, when reached, is
// exact (c = 0).  Returns the exact-as-possible change of the thrust.
__device__ __forceinline__ float rotor_advance(float& T, float& c, float y, float tmin, float tmax) {
  const float yc = y - c;
  float t = T + yc;
  float cn = (t - T) - yc;
  if (t > tmax) { t = tmax; cn = 0.f; }
  if (t < tmin) { t = tmin; cn = 0.f; }
  const float d = (t - T) - (cn - c);
  T = t;
  c = cn;
  return d;
}

// One classical RK4 step of the rotor model.  The stage thrusts are the exact
// saturating ramps at t, t + h/2 and t + h (T is not integrated); the
// thrusts (T, Tc: compensated, true value T - Tc) advance to the end of the
// step.  dp receives the position increment, dT2 the squared thrust change
// sum_s (T_s(t+h) - T_s(t))^2.
template <bool DRAG>
__device__ __forceinline__ void rk4_step_rotor(const ModelRegs& M, const RotorRegs& R, const StepConsts* sc,
                                               Quad& s, float qe, float T[4], float Tc[4], float u0, float u1,
                                               float u2, float u3, float h, float& dpx, float& dpy, float& dpz,
                                               float& dT2) {
  const float h2 = 0.5f * h, h4 = 0.25f * h;
  const float iml = lds4_volatile(&sc->c[1]).z;
  const float t0 = T[0] - Tc[0], t1 = T[1] - Tc[1], t2 = T[2] - Tc[2], t3 = T[3] - Tc[3];
  const float m0 = clampf(T[0] + (u0 * h2 - Tc[0]), R.tmin, R.tmax);
  const float m1 = clampf(T[1] + (u1 * h2 - Tc[1]), R.tmin, R.tmax);
  const float m2 = clampf(T[2] + (u2 * h2 - Tc[2]), R.tmin, R.tmax);
  const float m3 = clampf(T[3] + (u3 * h2 - Tc[3]), R.tmin, R.tmax);
  float e[4] = {T[0], T[1], T[2], T[3]}, ec[4] = {Tc[0], Tc[1], Tc[2], Tc[3]};
  const float d0 = rotor_advance(e[0], ec[0], u0 * h, R.tmin, R.tmax);
  const float d1 = rotor_advance(e[1], ec[1], u1 * h, R.tmin, R.tmax);
  const float d2 = rotor_advance(e[2], ec[2], u2 * h, R.tmin, R.tmax);
  const float d3 = rotor_advance(e[3], ec[3], u3 * h, R.tmin, R.tmax);
  const float e0 = e[0] - ec[0], e1 = e[1] - ec[1], e2 = e[2] - ec[2], e3 = e[3] - ec[3];
  float ac2, acg, bx, by, bz;
  float dqw, dqx, dqy, dqz, dwx, dwy, dwz, ax, ay, az;
  // stage 1 (start-of-step thrusts)
  rotor_forces(M, R, iml, t0, t1, t2, t3, ac2, acg, bx, by, bz);
  attitude_rate2_torque(M, bx, by, bz, s.qw, s.qx, s.qy, s.qz, s.wx, s.wy, s.wz, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, s.qw, s.qx, s.qy, s.qz, s.vx, s.vy, s.vz, ax, ay, az);
  else
    accel_nodrag(ac2, acg, s.qw, s.qx, s.qy, s.qz, ax, ay, az);
  float sqw = dqw, sqx = dqx, sqy = dqy, sqz = dqz, swx = dwx, swy = dwy, swz = dwz;
  float sax = ax, say = ay, saz = az;
  float pax = ax, pay = ay, paz = az;
  float vx2 = 0.f, vy2 = 0.f, vz2 = 0.f;
  // stages 2 and 3 (mid-step thrusts)
  rotor_forces(M, R, iml, m0, m1, m2, m3, ac2, acg, bx, by, bz);
  float qw2 = s.qw + h4 * dqw, qx2 = s.qx + h4 * dqx, qy2 = s.qy + h4 * dqy, qz2 = s.qz + h4 * dqz;
  float wx2 = s.wx + h2 * dwx, wy2 = s.wy + h2 * dwy, wz2 = s.wz + h2 * dwz;
  if (DRAG) { vx2 = s.vx + h2 * ax; vy2 = s.vy + h2 * ay; vz2 = s.vz + h2 * az; }
  attitude_rate2_torque(M, bx, by, bz, qw2, qx2, qy2, qz2, wx2, wy2, wz2, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, qw2, qx2, qy2, qz2, vx2, vy2, vz2, ax, ay, az);
  else
    accel_nodrag(ac2, acg, qw2, qx2, qy2, qz2, ax, ay, az);
  sqw += 2.f * dqw; sqx += 2.f * dqx; sqy += 2.f * dqy; sqz += 2.f * dqz;
  swx += 2.f * dwx; swy += 2.f * dwy; swz += 2.f * dwz;
  sax += 2.f * ax; say += 2.f * ay; saz += 2.f * az;
  pax += ax; pay += ay; paz += az;
  qw2 = s.qw + h4 * dqw; qx2 = s.qx + h4 * dqx; qy2 = s.qy + h4 * dqy; qz2 = s.qz + h4 * dqz;
  wx2 = s.wx + h2 * dwx; wy2 = s.wy + h2 * dwy; wz2 = s.wz + h2 * dwz;
  if (DRAG) { vx2 = s.vx + h2 * ax; vy2 = s.vy + h2 * ay; vz2 = s.vz + h2 * az; }
  attitude_rate2_torque(M, bx, by, bz, qw2, qx2, qy2, qz2, wx2, wy2, wz2, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, qw2, qx2, qy2, qz2, vx2, vy2, vz2, ax, ay, az);
  else
    accel_nodrag(ac2, acg, qw2, qx2, qy2, qz2, ax, ay, az);
  sqw += 2.f * dqw; sqx += 2.f * dqx; sqy += 2.f * dqy; sqz += 2.f * dqz;
  swx += 2.f * dwx; swy += 2.f * dwy; swz += 2.f * dwz;
  sax += 2.f * ax; say += 2.f * ay; saz += 2.f * az;
  pax += ax; pay += ay; paz += az;
  // stage 4 (end-of-step thrusts)
  rotor_forces(M, R, iml, e0, e1, e2, e3, ac2, acg, bx, by, bz);
  qw2 = s.qw + h2 * dqw; qx2 = s.qx + h2 * dqx; qy2 = s.qy + h2 * dqy; qz2 = s.qz + h2 * dqz;
  wx2 = s.wx + h * dwx; wy2 = s.wy + h * dwy; wz2 = s.wz + h * dwz;
  if (DRAG) { vx2 = s.vx + h * ax; vy2 = s.vy + h * ay; vz2 = s.vz + h * az; }
  attitude_rate2_torque(M, bx, by, bz, qw2, qx2, qy2, qz2, wx2, wy2, wz2, dqw, dqx, dqy, dqz, dwx, dwy, dwz);
  if (DRAG)
    accel_drag(M, ac2, acg, qw2, qx2, qy2, qz2, vx2, vy2, vz2, ax, ay, az);
  else
    accel_nodrag(ac2, acg, qw2, qx2, qy2, qz2, ax, ay, az);
  sqw += dqw; sqx += dqx; sqy += dqy; sqz += dqz;
  swx += dwx; swy += dwy; swz += dwz;
  sax += ax; say += ay; saz += az;
  // combine (the collective-thrust step's form; w compensated too: this
  // model has no rate loop, so rounding in w integrates undamped)
  const float4 c0 = lds4_volatile(&sc->c[0]), c1 = lds4_volatile(&sc->c[1]);
  dpx = h * s.vx + c0.z * pax;
  dpy = h * s.vy + c0.z * pay;
  dpz = h * s.vz + c0.z * paz;
  kahan_add(s.px, s.cpx, dpx);
  kahan_add(s.py, s.cpy, dpy);
  kahan_add(s.pz, s.cpz, dpz);
  s.cpx -= c0.w * pax;
  s.cpy -= c0.w * pay;
  s.cpz -= c0.w * paz;
  vel_advance(s.vx, s.cvx, sax, c0.x, c0.y);
  vel_advance(s.vy, s.cvy, say, c0.x, c0.y);
  vel_advance(s.vz, s.cvz, saz, c0.x, c0.y);
  vel_advance(s.wx, s.cwx, swx, c0.x, c0.y);
  vel_advance(s.wy, s.cwy, swy, c0.x, c0.y);
  vel_advance(s.wz, s.cwz, swz, c0.x, c0.y);
  quat_advance(s, qe, fmaf(c1.y, sqw, c1.x * sqw), fmaf(c1.y, sqx, c1.x * sqx), fmaf(c1.y, sqy, c1.x * sqy),
               fmaf(c1.y, sqz, c1.x * sqz));
  dT2 = d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    T[r] = e[r];
    Tc[r] = ec[r];
  }
}

// compensated position (hi - compensation)
__device__ __forceinline__ float pxt(const Quad& s) { return s.px - s.cpx; }
__device__ __forceinline__ float pyt(const Quad& s) { return s.py - s.cpy; }
__device__ __forceinline__ float pzt(const Quad& s) { return s.pz - s.cpz; }

__device__ __forceinline__ float limit_penalty(float wlim, float wmax, float zf, const Quad& s) {
  const float ex = fmaxf(fabsf(s.wx) - wmax, 0.f), ey = fmaxf(fabsf(s.wy) - wmax, 0.f),
              ez = fmaxf(fabsf(s.wz) - wmax, 0.f);
  const float e = fmaxf(zf - pzt(s), 0.f);
  return wlim * (ex * ex + ey * ey + ez * ez + e * e);
}


}  // namespace mppi
