// mppi_api.cu -- host side of the libmppi C ABI (see include/mppi.h).
//
// A handle owns one device slab: its solve descriptor, the resident controller
// state (nominal U*, Philox iteration, gate index, pass counts, previous x0,
// progress state) and the per-solve buffers (noise, costs, tile partials).
// Solves enqueue the kernels of mppi_kernels.cu on the caller's stream; u0 is
// written by the device into mapped pinned host memory, so a synchronous solve
// waits for one event and copies nothing.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mppi_device.cuh"
#include "mppi_launch.h"

using namespace mppi;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return fail(MPPI_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
// bytes allocated past the reference table: a bulk copy of its rows is
// rounded up to 16 bytes
constexpr int kRefPad = 64;

struct Slab {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = al256(off + bytes);
    return o;
  }
};

// pinned host memory the device writes u0 / status into
struct HostIO {
  float* u0 = nullptr;      // [n][5]
  int32_t* status = nullptr;
  float* x0 = nullptr;      // [n][13]
  double* t0 = nullptr;     // [n]
  float* d_u0 = nullptr;    // device aliases of the mapped buffers
  int32_t* d_status = nullptr;
  float* d_x0 = nullptr;
  double* d_t0 = nullptr;
  void* base = nullptr;
  int n = 0;
};

int hostio_alloc(HostIO& io, int n) {
  size_t bytes = al256(sizeof(float) * 5 * n) + al256(sizeof(int32_t) * n) + al256(sizeof(float) * 13 * n) +
                 al256(sizeof(double) * n);
  void* p = nullptr;
  if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
    return fail(MPPI_ERR_OOM, "cudaHostAlloc of %zu bytes failed", bytes);
  memset(p, 0, bytes);
  char* c = static_cast<char*>(p);
  io.base = p;
  io.n = n;
  io.u0 = reinterpret_cast<float*>(c);
  c += al256(sizeof(float) * 5 * n);
  io.status = reinterpret_cast<int32_t*>(c);
  c += al256(sizeof(int32_t) * n);
  io.x0 = reinterpret_cast<float*>(c);
  c += al256(sizeof(float) * 13 * n);
  io.t0 = reinterpret_cast<double*>(c);
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) return fail(MPPI_ERR_CUDA, "cudaHostGetDevicePointer failed");
  char* dc = static_cast<char*>(d);
  io.d_u0 = reinterpret_cast<float*>(dc);
  dc += al256(sizeof(float) * 5 * n);
  io.d_status = reinterpret_cast<int32_t*>(dc);
  dc += al256(sizeof(int32_t) * n);
  io.d_x0 = reinterpret_cast<float*>(dc);
  dc += al256(sizeof(float) * 13 * n);
  io.d_t0 = reinterpret_cast<double*>(dc);
  return MPPI_OK;
}

void hostio_free(HostIO& io) {
  if (io.base) cudaFreeHost(io.base);
  io = HostIO{};
}

}  // namespace

void mppi::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct mppi_s {
  mppi_model_t model;
  mppi_params_t params;
  int device = 0;
  int K_cap = 0, N_cap = 0, T_cap = 0, nu = 4, block = 128;
  int n_gates = 0, S = 0, T = 0;
  unsigned version = 1;
  SolveDesc hd;          // host copy of the descriptor
  SolveDesc* d_desc = nullptr;
  Tile* d_tiles = nullptr;
  int32_t* d_which = nullptr;  // [1] = 0 (nominal kernel work list)
  void* slab = nullptr;
  size_t slab_bytes = 0;
  HostIO io;
  cudaEvent_t ev_u0 = nullptr;
  bool ext_noise_pending = false;
  // MPPI_NOISEGEN_AHEAD: the noise buffer holds the normals of the state's
  // current iteration (drawn after the previous solve, recorded by ev_ahead)
  bool ahead_ready = false;
  cudaEvent_t ev_ahead = nullptr;
  bool ahead_pending = false;      // ev_ahead records a draw ...
  cudaStream_t ahead_stream = 0;   // ... enqueued on this stream
};

struct mppi_batch_s;
static std::mutex g_plan_mu;
static std::vector<mppi_batch_s*> g_plans;

struct mppi_batch_s {
  std::vector<mppi_handle> hs;
  std::vector<unsigned> versions;
  int n = 0;
  // mppi_solve_batch's cache (guarded by g_plan_mu): calls running this plan,
  // and whether it has left the cache (the last user then destroys it)
  int users = 0;
  bool evicted = false;
  SolveDesc* d_descs = nullptr;
  struct Group {
    int objective, bf16, block, gen, nom, rot;  // gen: MPPI_NOISEGEN_*; nom: nominal candidate; rot: rotor model
    uint32_t smem;
    int n_tiles;
    Tile* d_tiles;
    Tile* d_noise_tiles;  // the same tiles, for this group's own noise launch
  };
  std::vector<cudaStream_t> branch_streams;
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[8] = {};
  std::vector<Group> rollout_groups;
  struct NGroup {
    int bf16, block, nom, n_tiles;
    Tile* d_tiles;
  };
  std::vector<NGroup> noise_groups;
  int32_t* d_which = nullptr;
  int n_which = 0;
  // captured form: the rollout group (branch) that holds every gate-progress
  // solve runs the nominal rollouts right after its own rollout, so that they
  // overlap the other branches instead of following the join (-1: after it)
  int nominal_branch = -1;
  void* dev = nullptr;
  HostIO io;
  bool use_graph = false;
  bool branches = false;  // graph with one branch per rollout group
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev = nullptr;
  int kernels_per_solve = 0;  // kernels one launch of the sequence runs
  // second graph whose inputs/outputs are the plan's own device buffers
  // (the device-resident async path copies into / out of them)
  cudaGraph_t graph_dev = nullptr;
  cudaGraphExec_t exec_dev = nullptr;
  float* d_x0s = nullptr;
  double* d_t0s = nullptr;
  float* d_u0s = nullptr;
  // graphs captured on the caller's own device buffers: a call whose
  // (x0, t0, u0) pointers match one of them launches it with no copies
  struct DevExec {
    const float* x0;
    const double* t0;
    float* u0;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  };
  std::vector<DevExec> dev_execs;
};

// caller pointer sets a plan keeps graphs for; further sets use the copy path
constexpr size_t kMaxDevExecs = 4;

namespace {

int validate(const mppi_model_t* m, const mppi_params_t* p, const mppi_track_t* t) {
  if (!m || !p || !t) return fail(MPPI_ERR_ARG, "null model, params or track");
  if (m->kind != MPPI_MODEL_CTBR && m->kind != MPPI_MODEL_ROTOR_RATE)
    return fail(MPPI_ERR_ARG, "unknown model kind %d", m->kind);
  if (m->kind == MPPI_MODEL_ROTOR_RATE) {
    if (!(m->arm > 0) || !(m->c_tau >= 0) || !(m->thrust_max > m->thrust_min))
      return fail(MPPI_ERR_ARG, "rotor model needs arm > 0, c_tau >= 0 and thrust_max > thrust_min");
    if (p && p->noise_dtype != MPPI_NOISE_F32) return fail(MPPI_ERR_ARG, "the rotor model uses float32 noise storage");
  }
  if (!(m->mass > 0) || !(m->inertia[0] > 0) || !(m->inertia[1] > 0) || !(m->inertia[2] > 0))
    return fail(MPPI_ERR_ARG, "mass and inertia must be positive");
  if (p->K < 1 || p->N < 1 || p->N > MPPI_MAX_N) return fail(MPPI_ERR_ARG, "K=%d N=%d out of range", p->K, p->N);
  if (p->K_cap && p->K_cap < p->K) return fail(MPPI_ERR_ARG, "K_cap < K");
  if (p->N_cap && (p->N_cap < p->N || p->N_cap > MPPI_MAX_N)) return fail(MPPI_ERR_ARG, "N_cap out of range");
  if (!(p->dt > 0) || !(p->lambda > 0)) return fail(MPPI_ERR_ARG, "dt and lambda must be positive");
  if (p->objective < 0 || p->objective > 2) return fail(MPPI_ERR_ARG, "unknown objective %d", p->objective);
  if (p->noise_dtype != MPPI_NOISE_F32 && p->noise_dtype != MPPI_NOISE_BF16)
    return fail(MPPI_ERR_ARG, "unknown noise dtype");
  if (p->accum < 0 || p->accum > 2) return fail(MPPI_ERR_ARG, "unknown accumulation mode");
  if (p->noise_gen < MPPI_NOISEGEN_KERNEL || p->noise_gen > MPPI_NOISEGEN_AHEAD)
    return fail(MPPI_ERR_ARG, "unknown noise generation mode");
  if (p->noise_gen == MPPI_NOISEGEN_REGEN && p->noise_dtype != MPPI_NOISE_F32)
    return fail(MPPI_ERR_ARG, "regenerated noise is never stored: it has no bfloat16 form");
  if (p->nominal_sample != 0 && p->nominal_sample != 1) return fail(MPPI_ERR_ARG, "nominal_sample must be 0 or 1");
  if (p->warm_start != MPPI_WARM_SHIFT && p->warm_start != MPPI_WARM_KEEP)
    return fail(MPPI_ERR_ARG, "unknown warm start");
  int blk = p->block ? p->block : 128;
  if (blk < 32 || blk > rollout_max_block() || blk % 32)
    return fail(MPPI_ERR_ARG, "block %d must be a multiple of 32 in [32, %d]", blk, rollout_max_block());
  if (p->samples_per_thread < 0 || p->samples_per_thread > MPPI_MAX_SPT)
    return fail(MPPI_ERR_ARG, "samples_per_thread %d outside [0, %d]", p->samples_per_thread, MPPI_MAX_SPT);
  if (p->noise_gen == MPPI_NOISEGEN_SMEM) {
    const int tile = blk * (p->samples_per_thread ? p->samples_per_thread : 1);
    const int Nc = p->N_cap ? p->N_cap : p->N, Kc = p->K_cap ? p->K_cap : p->K;
    const int rows = p->objective == MPPI_OBJ_TRACK ? ref_rows_for(Nc, p->dt, t->dt_ref, t->T) : 0;
    const uint32_t need = rollout_smem_bytes(Nc, p->objective, t->S, tile, std::max(32, (Kc + tile - 1) / tile),
                                             MPPI_NOISEGEN_SMEM, rows);
    if (need > kRolloutSmemMax)
      return fail(MPPI_ERR_ARG, "noise kept in shared memory needs %u bytes per block, more than %u", need,
                  kRolloutSmemMax);
  }
  if (t->n_gates < 0 || t->n_gates > MPPI_MAX_GATES) return fail(MPPI_ERR_ARG, "n_gates out of range");
  if (p->objective == MPPI_OBJ_GATE && (t->n_gates < 1 || !t->gates))
    return fail(MPPI_ERR_ARG, "gate objective needs at least one gate");
  if (p->objective == MPPI_OBJ_CONTOUR && (t->S < 2 || !t->path || !(t->L > 0)))
    return fail(MPPI_ERR_ARG, "contouring needs a path table (S >= 2, L > 0)");
  if (p->objective == MPPI_OBJ_TRACK && (t->T < 2 || !t->ref || !(t->dt_ref > 0)))
    return fail(MPPI_ERR_ARG, "tracking needs a reference table (T >= 2, dt_ref > 0)");
  return MPPI_OK;
}

struct Sizes {
  size_t off_desc, off_st, off_U, off_prev, off_gates, off_gframes, off_path, off_ref, off_Z, off_Z5, off_J, off_info, off_pm,
      off_pS, off_pP, off_ticket, off_unew, off_passcnt, off_xref, total;
};

Sizes plan_sizes(const mppi_params_t* p, const mppi_track_t* t) {
  const int K_cap = p->K_cap ? p->K_cap : p->K;
  const int N_cap = p->N_cap ? p->N_cap : p->N;
  const int blk = p->block ? p->block : 128;
  const int T_cap = (K_cap + blk - 1) / blk;
  int sq = 1;
  while (sq * sq < T_cap) ++sq;
  const int Gn = 2 * sq + 16;  // >= n_groups_for(T) for every T <= T_cap
  const bool bf16 = p->noise_dtype == MPPI_NOISE_BF16;
  const bool five = p->objective == MPPI_OBJ_CONTOUR;
  const bool stored = p->noise_gen != MPPI_NOISEGEN_REGEN && p->noise_gen != MPPI_NOISEGEN_SMEM;
  Slab s;
  Sizes z;
  z.off_desc = s.take(sizeof(SolveDesc));
  z.off_st = s.take(sizeof(DevState));
  z.off_U = s.take(sizeof(float) * (N_cap * kNU + 8));
  z.off_prev = s.take(sizeof(int32_t) * (N_cap + 8));
  z.off_gates = s.take(sizeof(float) * 6 * std::max(1, t->n_gates));
  z.off_gframes = s.take(sizeof(GateF) * std::max(1, t->n_gates));
  z.off_path = s.take(sizeof(float) * 6 * std::max(1, t->S) + 64);
  z.off_ref = s.take(sizeof(float) * 13 * std::max(1, t->T) + kRefPad);
  z.off_Z = s.take(stored ? (size_t)N_cap * K_cap * (bf16 ? 8 : 16) : 16);
  z.off_Z5 = s.take(five && stored ? (size_t)N_cap * K_cap * (bf16 ? 2 : 4) : 16);
  z.off_J = s.take(sizeof(double) * K_cap);
  z.off_info = s.take(sizeof(int32_t) * K_cap);
  z.off_pm = s.take(sizeof(double) * (T_cap + Gn + 1));
  z.off_pS = s.take(sizeof(double) * (T_cap + Gn + 1));
  z.off_pP = s.take(sizeof(double) * (size_t)(T_cap + Gn + 1) * N_cap * kNU);
  z.off_ticket = s.take(sizeof(uint32_t) * (Gn + 2));
  z.off_unew = s.take(sizeof(float) * N_cap * kNU);
  z.off_passcnt = s.take(sizeof(int32_t) * (N_cap + 1));
  z.off_xref = s.take(sizeof(float) * 13 * (N_cap + 1));
  z.total = s.off;
  return z;
}

}  // namespace

// x as a (hi, lo) binary32 pair
static void split_pair(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// The RK4 weights h/6, h^2/6, h/12, the low part of 1/m and the rotor torque
// factors as (hi, lo) pairs, computed here in double (see StepConsts).
void mppi::fill_step_consts(const mppi_model_t& m, float dt, SolveDesc& d) {
  const double h = (double)dt;
  float a, b, c, e, f, g;
  split_pair(h / 6.0, a, b);
  split_pair(h * h / 6.0, c, e);
  split_pair(h / 12.0, f, g);
  d.stepc.c[0] = make_float4(a, b, c, e);
  float im, iml;
  split_pair(1.0 / (double)m.mass, im, iml);
  d.stepc.c[1] = make_float4(f, g, iml, 0.f);
  const double arm2 = (double)m.arm / sqrt(2.0);
  split_pair(arm2 / (double)m.inertia[0], d.kt[0][0], d.kt[0][1]);
  split_pair(arm2 / (double)m.inertia[1], d.kt[1][0], d.kt[1][1]);
  split_pair((double)m.c_tau / (double)m.inertia[2], d.kt[2][0], d.kt[2][1]);
}

void mppi::fill_model_params(const mppi_model_t& m, const mppi_params_t& p, int nu, SolveDesc& d) {
  fill_step_consts(m, p.dt, d);
  d.wait_ns = 200000000u;  // 0.2 s for a few KB of bulk copies
  d.wait_unreachable = 0;
  d.mass = m.mass;
  d.inv_mass = (float)(1.0 / (double)m.mass);
  d.gravity = m.gravity;
  d.k_omega = m.k_omega;
  const double Jx = m.inertia[0], Jy = m.inertia[1], Jz = m.inertia[2];
  d.gyro[0] = (float)((Jz - Jy) / Jx);
  d.gyro[1] = (float)((Jx - Jz) / Jy);
  d.gyro[2] = (float)((Jy - Jx) / Jz);
  for (int i = 0; i < 3; ++i) d.drag[i] = m.drag[i];
  d.has_drag = (m.drag[0] != 0.f || m.drag[1] != 0.f || m.drag[2] != 0.f) ? 1 : 0;
  for (int i = 0; i < kNU; ++i) {
    d.u_min[i] = m.u_min[i];
    d.u_max[i] = m.u_max[i];
    d.sigma[i] = p.sigma[i];
  }
  d.omega_max = m.omega_max;
  d.z_floor = m.z_floor;
  d.objective = p.objective;
  d.K = p.K;
  d.N = p.N;
  d.nu = nu;
  d.dt = p.dt;
  d.lambda = p.lambda;
  d.inv_lambda = (float)(1.0 / (double)p.lambda);
  d.seed = p.seed;
  d.drone_id = p.drone_id;
  d.noise_bf16 = p.noise_dtype == MPPI_NOISE_BF16;
  d.noise_gen = p.noise_gen;
  d.nominal_sample = p.nominal_sample ? 1 : 0;
  d.warm_keep = p.warm_start == MPPI_WARM_KEEP ? 1 : 0;
  d.spt = p.samples_per_thread > 0 ? p.samples_per_thread : 1;
  d.accum = p.accum;
  d.w_limit = p.w_limit;
  d.q_near = p.q_near;
  d.r_near2 = p.r_near * p.r_near;
  d.temporal_rule = p.temporal_rule;
  d.q_lag = p.q_lag;
  d.q_cont = p.q_cont;
  for (int i = 0; i < 3; ++i) d.q_omega[i] = p.q_omega[i];
  d.r_dv = p.r_dv;
  d.r_dthrust = p.r_dthrust;
  d.mu = p.mu;
  d.v_theta_max = p.v_theta_max;
  d.theta_back = p.theta_back;
  d.theta_ahead = p.theta_ahead;
  for (int i = 0; i < kNX; ++i) {
    d.Q[i] = p.Q[i];
    d.QN[i] = p.QN[i];
  }
  for (int i = 0; i < 4; ++i) d.R[i] = p.R[i];
  d.hover = m.mass * m.gravity;
  d.rotor = m.kind == MPPI_MODEL_ROTOR_RATE ? 1 : 0;
  d.arm2 = (float)((double)m.arm / sqrt(2.0));
  d.c_tau = m.c_tau;
  d.thrust_min = m.thrust_min;
  d.thrust_max = m.thrust_max;
  for (int i = 0; i < 3; ++i) d.inv_J[i] = (float)(1.0 / (double)m.inertia[i]);
}

namespace {

void fill_desc(mppi_handle h) {
  fill_model_params(h->model, h->params, h->nu, h->hd);
  SolveDesc& d = h->hd;
  d.N_cap = h->N_cap;
  d.block = h->block;
  d.n_tiles = (h->params.K + tile_samples(d) - 1) / tile_samples(d);
  d.ext_noise = 0;
}

int upload_tiles(mppi_handle h) {
  const int T = h->hd.n_tiles;
  std::vector<Tile> tl(T);
  for (int i = 0; i < T; ++i) tl[i] = Tile{0, i * tile_samples(h->hd)};
  CU(cudaMemcpy(h->d_tiles, tl.data(), sizeof(Tile) * T, cudaMemcpyHostToDevice));
  return MPPI_OK;
}

// initial nominal: hover thrust (collective-thrust model) or zero rotor-thrust rates
void fill_hover(const mppi_handle h, std::vector<float>& U) {
  U.assign((size_t)h->N_cap * kNU + 8, 0.f);
  if (h->model.kind == MPPI_MODEL_ROTOR_RATE) return;
  for (int k = 0; k < h->N_cap; ++k) U[(size_t)k * kNU] = h->model.mass * h->model.gravity;
}

uint32_t merge_cap(int n_tiles) { return (uint32_t)std::max(n_tiles, 32); }

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* mppi_last_error(void) { return g_err.c_str(); }
const char* mppi_version(void) { return "libmppi 1.0 (sm_103a)"; }
uint64_t mppi_kernel_launches(void) { return (uint64_t)launches_so_far(); }

int mppi_abi_sizes(size_t out[3]) {
  if (!out) return fail(MPPI_ERR_ARG, "null argument");
  out[0] = sizeof(mppi_model_t);
  out[1] = sizeof(mppi_params_t);
  out[2] = sizeof(mppi_track_t);
  return MPPI_OK;
}

int mppi_default_model(mppi_model_t* m) {
  if (!m) return fail(MPPI_ERR_ARG, "null model");
  memset(m, 0, sizeof *m);
  m->kind = MPPI_MODEL_CTBR;
  m->mass = 0.85f;
  m->inertia[0] = 0.0025f;
  m->inertia[1] = 0.0025f;
  m->inertia[2] = 0.0043f;
  m->gravity = 9.81f;
  m->k_omega = 20.f;
  const float lo[5] = {0.f, -10.f, -10.f, -10.f, -20.f};
  const float hi[5] = {(float)(4.0 * 0.85 * 9.81), 10.f, 10.f, 10.f, 20.f};
  for (int i = 0; i < 5; ++i) {
    m->u_min[i] = lo[i];
    m->u_max[i] = hi[i];
  }
  m->omega_max = 10.f;
  m->z_floor = 0.f;
  m->arm = 0.15f;
  m->c_tau = 0.01f;
  m->thrust_min = 0.f;
  m->thrust_max = 10.f;
  return MPPI_OK;
}

int mppi_default_params(mppi_params_t* p, int32_t objective, int32_t K, int32_t N, float dt) {
  if (!p) return fail(MPPI_ERR_ARG, "null params");
  memset(p, 0, sizeof *p);
  p->objective = objective;
  p->K = K;
  p->N = N;
  p->dt = dt;
  p->lambda = 1.f;
  const float sg[5] = {(float)(0.3 * 0.85 * 9.81), 1.f, 1.f, 1.f, 5.f};
  for (int i = 0; i < 5; ++i) p->sigma[i] = sg[i];
  p->w_limit = 1000.f;
  p->q_near = 0.05f;
  p->r_near = 1.5f;
  p->temporal_rule = MPPI_RULE_TIME_ALIGNED;
  p->q_lag = 1.f;
  p->q_cont = 10.f;
  for (int i = 0; i < 3; ++i) p->q_omega[i] = 0.001f;
  p->r_dv = 0.001f;
  p->r_dthrust = 0.001f;
  p->mu = 0.1f;
  p->v_theta_max = 20.f;
  p->theta_back = 2.f;
  p->theta_ahead = 10.f;
  for (int i = 0; i < 13; ++i) {
    const float q = i < 3 ? 10.f : i < 6 ? 0.1f : i < 10 ? 1.f : 0.01f;
    p->Q[i] = q;
    p->QN[i] = 2.f * q;
  }
  p->R[0] = 0.001f;
  p->R[1] = p->R[2] = p->R[3] = 0.01f;
  p->noise_dtype = MPPI_NOISE_F32;
  p->accum = MPPI_ACC_KAHAN32;
  p->block = 128;
  p->samples_per_thread = 1;
  return MPPI_OK;
}

int mppi_estimate_bytes(const mppi_params_t* params, const mppi_track_t* track, size_t* bytes) {
  if (!params || !track || !bytes) return fail(MPPI_ERR_ARG, "null argument");
  *bytes = plan_sizes(params, track).total;
  return MPPI_OK;
}

int mppi_create(const mppi_model_t* model, const mppi_params_t* params, const mppi_track_t* track,
                mppi_handle* out) {
  if (!out) return fail(MPPI_ERR_ARG, "null output handle");
  *out = nullptr;
  int rc = validate(model, params, track);
  if (rc) return rc;
  {
    static std::mutex mu;
    static std::vector<int> configured;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(configured.begin(), configured.end(), dev) == configured.end()) {
      CU(configure_kernels());
      configured.push_back(dev);
    }
  }
  mppi_handle h = new mppi_s();
  h->model = *model;
  h->params = *params;
  CU(cudaGetDevice(&h->device));
  h->block = params->block ? params->block : 128;
  h->params.block = h->block;
  h->K_cap = params->K_cap ? params->K_cap : params->K;
  h->N_cap = params->N_cap ? params->N_cap : params->N;
  h->T_cap = (h->K_cap + h->block - 1) / h->block;
  h->nu = params->objective == MPPI_OBJ_CONTOUR ? 5 : 4;
  h->n_gates = track->n_gates;
  h->S = track->S;
  h->T = track->T;
  const Sizes z = plan_sizes(&h->params, track);
  h->slab_bytes = z.total;
  if (cudaMalloc(&h->slab, z.total) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(MPPI_ERR_OOM, "cudaMalloc of %zu bytes failed", z.total);
  }
  char* b = static_cast<char*>(h->slab);
  if (cudaMemset(h->slab, 0, z.total) != cudaSuccess) {
    mppi_destroy(h);
    return fail(MPPI_ERR_CUDA, "cudaMemset failed");
  }
  fill_desc(h);
  SolveDesc& d = h->hd;
  h->d_desc = reinterpret_cast<SolveDesc*>(b + z.off_desc);
  d.st = reinterpret_cast<DevState*>(b + z.off_st);
  d.U = reinterpret_cast<float*>(b + z.off_U);
  d.prevcnt = reinterpret_cast<int32_t*>(b + z.off_prev);
  d.gates = reinterpret_cast<float*>(b + z.off_gates);
  d.n_gates = track->n_gates;
  d.closed = track->closed ? 1 : 0;
  d.path = reinterpret_cast<float*>(b + z.off_path);
  d.S = track->S;
  d.L = track->L;
  d.ds = track->S > 0 ? (float)((double)track->L / track->S) : 1.f;
  d.inv_ds = track->S > 0 ? (float)((double)track->S / track->L) : 1.f;
  d.ref = reinterpret_cast<float*>(b + z.off_ref);
  d.T = track->T;
  d.dt_ref = track->dt_ref;
  d.gframes = reinterpret_cast<const GateF*>(b + z.off_gframes);
  d.ref_rows = d.objective == MPPI_OBJ_TRACK ? ref_rows_for(h->N_cap, d.dt, d.dt_ref, d.T) : 0;
  d.ref_pad = kRefPad;
  const bool bf16 = d.noise_bf16,
             stored = d.noise_gen != MPPI_NOISEGEN_REGEN && d.noise_gen != MPPI_NOISEGEN_SMEM;
  d.Z4 = (stored && !bf16) ? reinterpret_cast<float4*>(b + z.off_Z) : nullptr;
  d.Zb = (stored && bf16) ? reinterpret_cast<uint2*>(b + z.off_Z) : nullptr;
  d.Z5 = (stored && !bf16 && h->nu == 5) ? reinterpret_cast<float*>(b + z.off_Z5) : nullptr;
  d.Z5b = (stored && bf16 && h->nu == 5) ? reinterpret_cast<__nv_bfloat16*>(b + z.off_Z5) : nullptr;
  d.J = reinterpret_cast<double*>(b + z.off_J);
  d.info = reinterpret_cast<int32_t*>(b + z.off_info);
  d.part_m = reinterpret_cast<double*>(b + z.off_pm);
  d.part_S = reinterpret_cast<double*>(b + z.off_pS);
  d.part_P = reinterpret_cast<double*>(b + z.off_pP);
  d.ticket = reinterpret_cast<uint32_t*>(b + z.off_ticket);
  d.unew = reinterpret_cast<float*>(b + z.off_unew);
  d.passcnt = reinterpret_cast<int32_t*>(b + z.off_passcnt);
  d.xref = reinterpret_cast<float*>(b + z.off_xref);

  auto cleanup = [&](int code) {
    mppi_destroy(h);
    return code;
  };
  // track tables
  if (track->n_gates > 0 && track->gates &&
      cudaMemcpy((void*)d.gates, track->gates, sizeof(float) * 6 * track->n_gates, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload of gates failed"));
  if (track->n_gates > 0 && track->gates &&
      (launch_gate_frames(d.gates, track->n_gates, const_cast<GateF*>(d.gframes), 0) != cudaSuccess ||
       cudaStreamSynchronize(0) != cudaSuccess))
    return cleanup(fail(MPPI_ERR_CUDA, "gate frames failed"));
  if (track->S > 0 && track->path &&
      cudaMemcpy((void*)d.path, track->path, sizeof(float) * 6 * track->S, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload of path failed"));
  if (track->T > 0 && track->ref &&
      cudaMemcpy((void*)d.ref, track->ref, sizeof(float) * 13 * track->T, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload of reference failed"));
  // resident state: hover nominal, zero counts
  std::vector<float> U;
  fill_hover(h, U);
  if (cudaMemcpy(d.U, U.data(), sizeof(float) * U.size(), cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload of nominal failed"));
  DevState st;
  memset(&st, 0, sizeof st);
  st.c_last = model->mass * model->gravity;
  st.status = MPPI_OK;
  if (cudaMemcpy(d.st, &st, sizeof st, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload of state failed"));
  if (cudaMemcpy(h->d_desc, &d, sizeof d, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload of descriptor failed"));
  if (cudaMalloc(&h->d_tiles, sizeof(Tile) * h->T_cap + sizeof(int32_t) * 4) != cudaSuccess)
    return cleanup(fail(MPPI_ERR_OOM, "tile table allocation failed"));
  h->d_which = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(h->d_tiles) + sizeof(Tile) * h->T_cap);
  int zero = 0;
  if (cudaMemcpy(h->d_which, &zero, sizeof zero, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "upload failed"));
  if ((rc = upload_tiles(h))) return cleanup(rc);
  if ((rc = hostio_alloc(h->io, 1))) return cleanup(rc);
  if (cudaEventCreateWithFlags(&h->ev_u0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_ahead, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(MPPI_ERR_CUDA, "event creation failed"));
  *out = h;
  return MPPI_OK;
}

int mppi_destroy(mppi_handle h) {
  if (!h) return MPPI_OK;
  {
    // cached batch plans that reference this handle are dropped with it
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (size_t i = 0; i < g_plans.size();) {
      mppi_batch p = g_plans[i];
      if (std::find(p->hs.begin(), p->hs.end(), h) != p->hs.end()) {
        g_plans.erase(g_plans.begin() + i);
        if (p->users == 0)
          mppi_batch_destroy(p);
        else
          p->evicted = true;
      } else {
        ++i;
      }
    }
  }
  if (h->ev_u0) cudaEventDestroy(h->ev_u0);
  if (h->ev_ahead) cudaEventDestroy(h->ev_ahead);
  hostio_free(h->io);
  if (h->d_tiles) cudaFree(h->d_tiles);
  if (h->slab) cudaFree(h->slab);
  delete h;
  return MPPI_OK;
}

int mppi_device_bytes(mppi_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(MPPI_ERR_ARG, "null argument");
  *bytes = h->slab_bytes + sizeof(Tile) * h->T_cap;
  return MPPI_OK;
}

int mppi_set_shape(mppi_handle h, int32_t K, int32_t N) {
  if (!h) return fail(MPPI_ERR_ARG, "null handle");
  if (K < 1 || K > h->K_cap || N < 1 || N > h->N_cap)
    return fail(MPPI_ERR_ARG, "shape K=%d N=%d outside the capacity K<=%d N<=%d", K, N, h->K_cap, h->N_cap);
  h->params.K = K;
  h->params.N = N;
  h->hd.K = K;
  h->hd.N = N;
  h->hd.n_tiles = (K + tile_samples(h->hd) - 1) / tile_samples(h->hd);
  CU(cudaMemcpy(h->d_desc, &h->hd, sizeof h->hd, cudaMemcpyHostToDevice));
  int rc = upload_tiles(h);
  if (rc) return rc;
  h->ahead_ready = false;  // the normals drawn ahead have the old shape
  ++h->version;
  return MPPI_OK;
}

// MPPI_NOISEGEN_AHEAD: orders stream s after the handle's pending draw, which
// may sit on another stream.  A capturing stream is left alone: its graph
// replays in stream order, and an event recorded outside the capture cannot
// be waited on inside it.
static int wait_ahead(mppi_handle h, cudaStream_t s) {
  if (h->hd.noise_gen != MPPI_NOISEGEN_AHEAD) return MPPI_OK;
  if (!h->ahead_pending || h->ahead_stream == s) return MPPI_OK;  // nothing to wait for, or in order
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusNone) CU(cudaStreamWaitEvent(s, h->ev_ahead, 0));
  return MPPI_OK;
}

static int enqueue_single(mppi_handle h, const LaunchIO& io, cudaStream_t s) {
  const SolveDesc& d = h->hd;
  int gen = 0;  // caller noise is already stored: the rollout loads it
  const bool ahead = d.noise_gen == MPPI_NOISEGEN_AHEAD;
  int rc = wait_ahead(h, s);
  if (rc) return rc;
  if (h->ext_noise_pending) {
    h->ext_noise_pending = false;
  } else if (ahead) {
    // drawn after the previous solve, unless something moved the counters since
    if (!h->ahead_ready)
      CU(launch_noise(h->d_desc, h->d_tiles, d.n_tiles, h->block, d.noise_bf16, s, d.nominal_sample, d.N));
  } else if (d.noise_gen != MPPI_NOISEGEN_KERNEL) {
    gen = d.noise_gen;
  } else {
    CU(launch_noise(h->d_desc, h->d_tiles, d.n_tiles, h->block, d.noise_bf16, s, d.nominal_sample, d.N));
  }
  const uint32_t smem =
      rollout_smem_bytes(d.N, d.objective, d.S, tile_samples(d), merge_cap(d.n_tiles), gen, d.ref_rows);
  CU(launch_rollout(d.objective, d.noise_bf16, h->d_desc, h->d_tiles, d.n_tiles, h->block, smem, io, s, gen,
                    d.rotor));
  h->ahead_ready = false;
  return MPPI_OK;
}

// MPPI_NOISEGEN_AHEAD, after the solve's own kernels: the normals of the next
// iteration (the counter the solve advanced), off the path to u0
static int draw_ahead(mppi_handle h, cudaStream_t s) {
  const SolveDesc& d = h->hd;
  if (d.noise_gen != MPPI_NOISEGEN_AHEAD) return MPPI_OK;
  CU(launch_noise(h->d_desc, h->d_tiles, d.n_tiles, h->block, d.noise_bf16, s, d.nominal_sample, d.N));
  CU(cudaEventRecord(h->ev_ahead, s));
  h->ahead_ready = true;
  h->ahead_pending = true;
  h->ahead_stream = s;
  return MPPI_OK;
}

int mppi_solve(mppi_handle h, const float x0[13], double t0, void* stream, float u0_out[5]) {
  if (!h || !x0 || !u0_out) return fail(MPPI_ERR_ARG, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LaunchIO io;
  memset(&io, 0, sizeof io);
  io.x0 = nullptr;
  io.t0 = nullptr;
  for (int i = 0; i < kNX; ++i) io.x0v[i] = x0[i];
  io.t0v = t0;
  io.u0 = h->io.d_u0;
  io.status = h->io.d_status;
  int rc = enqueue_single(h, io, s);
  if (rc) return rc;
  CU(cudaEventRecord(h->ev_u0, s));
  if (h->hd.objective == MPPI_OBJ_GATE) CU(launch_nominal(h->d_desc, h->d_which, 1, s));
  if ((rc = draw_ahead(h, s))) return rc;
  CU(cudaEventSynchronize(h->ev_u0));
  for (int i = 0; i < kNU; ++i) u0_out[i] = ((volatile float*)h->io.u0)[i];
  const int st = ((volatile int32_t*)h->io.status)[0];
  if (st == MPPI_ERR_TIMEOUT) return fail(MPPI_ERR_TIMEOUT, "a bounded wait for the bulk copies gave up");
  if (st == MPPI_WARN_DEGENERATE) return fail(MPPI_WARN_DEGENERATE, "every sample cost was non-finite");
  return MPPI_OK;
}

int mppi_set_copy_wait(mppi_handle h, uint32_t limit_ns, int32_t unreachable) {
  if (!h) return fail(MPPI_ERR_ARG, "null handle");
  h->hd.wait_ns = limit_ns;
  h->hd.wait_unreachable = unreachable ? 1 : 0;
  CU(cudaMemcpy(h->d_desc, &h->hd, sizeof h->hd, cudaMemcpyHostToDevice));
  ++h->version;
  return MPPI_OK;
}

int mppi_solve_async(mppi_handle h, const float* d_x0, double t0, void* stream, float* d_u0) {
  if (!h || !d_x0 || !d_u0) return fail(MPPI_ERR_ARG, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LaunchIO io;
  memset(&io, 0, sizeof io);
  io.x0 = d_x0;
  io.t0 = nullptr;
  io.t0v = t0;
  io.u0 = d_u0;
  io.status = nullptr;
  int rc = enqueue_single(h, io, s);
  if (rc) return rc;
  if (h->hd.objective == MPPI_OBJ_GATE) CU(launch_nominal(h->d_desc, h->d_which, 1, s));
  return draw_ahead(h, s);
}

// ---------------------------------------------------------------------------
// state access
// ---------------------------------------------------------------------------
int mppi_get_nominal(mppi_handle h, float* U) {
  if (!h || !U) return fail(MPPI_ERR_ARG, "null argument");
  CU(cudaMemcpy(U, h->hd.U, sizeof(float) * h->hd.N * kNU, cudaMemcpyDeviceToHost));
  return MPPI_OK;
}
int mppi_get_unew(mppi_handle h, float* U) {
  if (!h || !U) return fail(MPPI_ERR_ARG, "null argument");
  CU(cudaMemcpy(U, h->hd.unew, sizeof(float) * h->hd.N * kNU, cudaMemcpyDeviceToHost));
  return MPPI_OK;
}
int mppi_get_costs(mppi_handle h, double* J) {
  if (!h || !J) return fail(MPPI_ERR_ARG, "null argument");
  // the device keeps each cost as its compensated (hi, lo) binary32 pair
  CU(cudaMemcpy(J, h->hd.J, sizeof(double) * h->hd.K, cudaMemcpyDeviceToHost));
  for (int m = 0; m < h->hd.K; ++m) {
    float pair[2];
    memcpy(pair, &J[m], sizeof pair);
    J[m] = (double)pair[0] + (double)pair[1];
  }
  return MPPI_OK;
}
int mppi_get_sample_info(mppi_handle h, int32_t* npass, int32_t* first_pass) {
  if (!h) return fail(MPPI_ERR_ARG, "null handle");
  std::vector<int32_t> info(h->hd.K);
  CU(cudaMemcpy(info.data(), h->hd.info, sizeof(int32_t) * h->hd.K, cudaMemcpyDeviceToHost));
  for (int m = 0; m < h->hd.K; ++m) {
    if (npass) npass[m] = info[m] & 0xFFFF;
    if (first_pass) first_pass[m] = (info[m] >> 16) - 1;
  }
  return MPPI_OK;
}
int mppi_get_noise(mppi_handle h, float* Z) {
  if (!h || !Z) return fail(MPPI_ERR_ARG, "null argument");
  const SolveDesc& d = h->hd;
  if (d.noise_gen == MPPI_NOISEGEN_REGEN || d.noise_gen == MPPI_NOISEGEN_SMEM)
    return fail(MPPI_ERR_ARG, "this handle keeps no noise in device memory");
  if (d.noise_gen == MPPI_NOISEGEN_AHEAD) CU(cudaEventSynchronize(h->ev_ahead));
  const size_t nk = (size_t)d.N * d.K;
  std::vector<float> z4(nk * 4), z5(h->nu == 5 ? nk : 0);
  if (d.noise_bf16) {
    std::vector<uint16_t> b(nk * 4), b5(h->nu == 5 ? nk : 0);
    CU(cudaMemcpy(b.data(), d.Zb, nk * 8, cudaMemcpyDeviceToHost));
    if (h->nu == 5) CU(cudaMemcpy(b5.data(), d.Z5b, nk * 2, cudaMemcpyDeviceToHost));
    auto widen = [](uint16_t v) {
      uint32_t w = (uint32_t)v << 16;
      float f;
      memcpy(&f, &w, 4);
      return f;
    };
    for (size_t i = 0; i < nk * 4; ++i) z4[i] = widen(b[i]);
    for (size_t i = 0; i < z5.size(); ++i) z5[i] = widen(b5[i]);
  } else {
    CU(cudaMemcpy(z4.data(), d.Z4, nk * 16, cudaMemcpyDeviceToHost));
    if (h->nu == 5) CU(cudaMemcpy(z5.data(), d.Z5, nk * 4, cudaMemcpyDeviceToHost));
  }
  for (size_t i = 0; i < nk; ++i) {
    for (int j = 0; j < 4; ++j) Z[i * 5 + j] = z4[i * 4 + j];
    Z[i * 5 + 4] = h->nu == 5 ? z5[i] : 0.f;
  }
  return MPPI_OK;
}
int mppi_get_passcnt(mppi_handle h, int32_t* passcnt) {
  if (!h || !passcnt) return fail(MPPI_ERR_ARG, "null argument");
  CU(cudaMemcpy(passcnt, h->hd.passcnt, sizeof(int32_t) * (h->hd.N + 1), cudaMemcpyDeviceToHost));
  return MPPI_OK;
}
int mppi_get_info(mppi_handle h, int32_t info[4]) {
  if (!h || !info) return fail(MPPI_ERR_ARG, "null argument");
  DevState st;
  CU(cudaMemcpy(&st, h->hd.st, sizeof st, cudaMemcpyDeviceToHost));
  info[0] = st.gate0;
  info[1] = st.status;
  info[2] = (int32_t)st.iter;
  info[3] = st.gate;
  return MPPI_OK;
}
int mppi_get_solve_scalars(mppi_handle h, double out[4]) {
  if (!h || !out) return fail(MPPI_ERR_ARG, "null argument");
  DevState st;
  CU(cudaMemcpy(&st, h->hd.st, sizeof st, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) out[i] = st.scal[i];
  return MPPI_OK;
}
int mppi_get_xref(mppi_handle h, float* xref) {
  if (!h || !xref) return fail(MPPI_ERR_ARG, "null argument");
  CU(cudaMemcpy(xref, h->hd.xref, sizeof(float) * 13 * (h->hd.N + 1), cudaMemcpyDeviceToHost));
  return MPPI_OK;
}

// serialised state: header, DevState, U [N_cap][5], prevcnt [N_cap]
struct StateHeader {
  uint32_t magic, version, N_cap, nu;
};
static const uint32_t kMagic = 0x4D505049u;  // "MPPI"

int mppi_export_state(mppi_handle h, void* buf, size_t* size) {
  if (!h || !size) return fail(MPPI_ERR_ARG, "null argument");
  const size_t need = sizeof(StateHeader) + sizeof(DevState) + sizeof(float) * h->N_cap * kNU +
                      sizeof(int32_t) * h->N_cap;
  if (!buf) {
    *size = need;
    return MPPI_OK;
  }
  if (*size < need) return fail(MPPI_ERR_ARG, "buffer of %zu bytes, need %zu", *size, need);
  char* c = static_cast<char*>(buf);
  StateHeader hd{kMagic, 1u, (uint32_t)h->N_cap, (uint32_t)h->nu};
  memcpy(c, &hd, sizeof hd);
  c += sizeof hd;
  CU(cudaMemcpy(c, h->hd.st, sizeof(DevState), cudaMemcpyDeviceToHost));
  c += sizeof(DevState);
  CU(cudaMemcpy(c, h->hd.U, sizeof(float) * h->N_cap * kNU, cudaMemcpyDeviceToHost));
  c += sizeof(float) * h->N_cap * kNU;
  CU(cudaMemcpy(c, h->hd.prevcnt, sizeof(int32_t) * h->N_cap, cudaMemcpyDeviceToHost));
  *size = need;
  return MPPI_OK;
}

int mppi_import_state(mppi_handle h, const void* buf, size_t size) {
  if (!h || !buf) return fail(MPPI_ERR_ARG, "null argument");
  const size_t need = sizeof(StateHeader) + sizeof(DevState) + sizeof(float) * h->N_cap * kNU +
                      sizeof(int32_t) * h->N_cap;
  if (size < need) return fail(MPPI_ERR_ARG, "state blob of %zu bytes, need %zu", size, need);
  const char* c = static_cast<const char*>(buf);
  StateHeader hd;
  memcpy(&hd, c, sizeof hd);
  if (hd.magic != kMagic || hd.version != 1u || (int)hd.N_cap != h->N_cap || (int)hd.nu != h->nu)
    return fail(MPPI_ERR_ARG, "state blob does not match this handle");
  c += sizeof hd;
  DevState st;
  memcpy(&st, c, sizeof st);
  if (st.gate < 0) return fail(MPPI_ERR_ARG, "state blob has a negative gate index");
  CU(cudaMemcpy(h->hd.st, c, sizeof(DevState), cudaMemcpyHostToDevice));
  c += sizeof(DevState);
  CU(cudaMemcpy(h->hd.U, c, sizeof(float) * h->N_cap * kNU, cudaMemcpyHostToDevice));
  c += sizeof(float) * h->N_cap * kNU;
  CU(cudaMemcpy(h->hd.prevcnt, c, sizeof(int32_t) * h->N_cap, cudaMemcpyHostToDevice));
  h->ahead_ready = false;  // the iteration counter may have moved
  return MPPI_OK;
}

int mppi_set_gate_index(mppi_handle h, int32_t gate) {
  if (!h) return fail(MPPI_ERR_ARG, "null handle");
  if (gate < 0) return fail(MPPI_ERR_ARG, "gate index %d is negative", (int)gate);
  CU(cudaMemcpy(&h->hd.st->gate, &gate, sizeof gate, cudaMemcpyHostToDevice));
  return MPPI_OK;
}

int mppi_set_rotor_thrusts(mppi_handle h, const float T[4]) {
  if (!h || !T) return fail(MPPI_ERR_ARG, "null argument");
  if (!h->hd.rotor) return fail(MPPI_ERR_ARG, "not a rotor-model handle");
  DevState st;
  CU(cudaMemcpy(&st, h->hd.st, sizeof st, cudaMemcpyDeviceToHost));
  for (int r = 0; r < 4; ++r) st.rotor[r] = T[r];
  st.has_rotor = 1;
  CU(cudaMemcpy(h->hd.st, &st, sizeof st, cudaMemcpyHostToDevice));
  return MPPI_OK;
}

int mppi_get_rotor_thrusts(mppi_handle h, float T[4]) {
  if (!h || !T) return fail(MPPI_ERR_ARG, "null argument");
  if (!h->hd.rotor) return fail(MPPI_ERR_ARG, "not a rotor-model handle");
  DevState st;
  CU(cudaMemcpy(&st, h->hd.st, sizeof st, cudaMemcpyDeviceToHost));
  for (int r = 0; r < 4; ++r) T[r] = st.has_rotor ? st.rotor[r] : 0.25f * h->hd.hover;
  return MPPI_OK;
}

int mppi_set_noise(mppi_handle h, const void* d_Z, const void* d_Z5, void* stream) {
  if (!h || !d_Z) return fail(MPPI_ERR_ARG, "null argument");
  if (h->nu == 5 && !d_Z5) return fail(MPPI_ERR_ARG, "contouring needs the 5th noise column");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const SolveDesc& d = h->hd;
  if (d.noise_gen == MPPI_NOISEGEN_REGEN || d.noise_gen == MPPI_NOISEGEN_SMEM)
    return fail(MPPI_ERR_ARG, "this handle has no noise buffer");
  int rc = wait_ahead(h, s);
  if (rc) return rc;
  const size_t nk = (size_t)d.N * d.K;
  const size_t el = d.noise_bf16 ? 2 : 4;
  void* z4 = d.noise_bf16 ? (void*)d.Zb : (void*)d.Z4;
  void* z5 = d.noise_bf16 ? (void*)d.Z5b : (void*)d.Z5;
  CU(cudaMemcpyAsync(z4, d_Z, nk * 4 * el, cudaMemcpyDeviceToDevice, s));
  if (h->nu == 5) CU(cudaMemcpyAsync(z5, d_Z5, nk * el, cudaMemcpyDeviceToDevice, s));
  if (d.nominal_sample) {
    // the nominal candidate carries no perturbation: zero its column
    CU(cudaMemset2DAsync(z4, (size_t)d.K * 4 * el, 0, 4 * el, d.N, s));
    if (h->nu == 5) CU(cudaMemset2DAsync(z5, (size_t)d.K * el, 0, el, d.N, s));
  }
  h->ext_noise_pending = true;
  return MPPI_OK;
}

int mppi_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int32_t n,
                uint32_t* d_out, void* stream) {
  if (n < 0 || (n > 0 && !d_out)) return fail(MPPI_ERR_ARG, "bad arguments");
  CU(launch_philox(k0, k1, c0, c1, c2, c3, n, d_out, static_cast<cudaStream_t>(stream)));
  return MPPI_OK;
}

int mppi_normals(uint32_t seed, uint32_t drone, uint32_t k, uint32_t it, uint32_t blk, int32_t n, float* d_out,
                 void* stream) {
  if (n < 0 || (n > 0 && !d_out)) return fail(MPPI_ERR_ARG, "bad arguments");
  CU(launch_normals(seed, drone, k, it, blk, n, d_out, static_cast<cudaStream_t>(stream)));
  return MPPI_OK;
}

static int rollout_states_impl(const mppi_model_t* model, float dt, int32_t N, int32_t B, const float* d_x0,
                               const float* d_U, float* d_X, void* stream, const float* d_T0, float* d_T) {
  SolveDesc md;
  memset(&md, 0, sizeof md);
  md.rotor = model->kind == MPPI_MODEL_ROTOR_RATE ? 1 : 0;
  md.arm2 = (float)((double)model->arm / sqrt(2.0));
  md.c_tau = model->c_tau;
  md.thrust_min = model->thrust_min;
  md.thrust_max = model->thrust_max;
  for (int i = 0; i < 3; ++i) md.inv_J[i] = (float)(1.0 / (double)model->inertia[i]);
  md.inv_mass = (float)(1.0 / (double)model->mass);
  md.gravity = model->gravity;
  md.k_omega = model->k_omega;
  const double Jx = model->inertia[0], Jy = model->inertia[1], Jz = model->inertia[2];
  md.gyro[0] = (float)((Jz - Jy) / Jx);
  md.gyro[1] = (float)((Jx - Jz) / Jy);
  md.gyro[2] = (float)((Jy - Jx) / Jz);
  for (int i = 0; i < 3; ++i) md.drag[i] = model->drag[i];
  md.has_drag = (model->drag[0] != 0.f || model->drag[1] != 0.f || model->drag[2] != 0.f) ? 1 : 0;
  fill_step_consts(*model, dt, md);
  CU(launch_rollout_states(md, dt, N, B, d_x0, d_U, d_X, static_cast<cudaStream_t>(stream), d_T0, d_T));
  return MPPI_OK;
}

int mppi_rollout_states(const mppi_model_t* model, float dt, int32_t N, int32_t B, const float* d_x0,
                        const float* d_U, float* d_X, void* stream) {
  if (!model || N < 1 || B < 0 || (B > 0 && (!d_x0 || !d_U || !d_X))) return fail(MPPI_ERR_ARG, "bad arguments");
  if (model->kind != MPPI_MODEL_CTBR) return fail(MPPI_ERR_ARG, "rotor model: use mppi_rollout_states_rotor");
  return rollout_states_impl(model, dt, N, B, d_x0, d_U, d_X, stream, nullptr, nullptr);
}

int mppi_rollout_states_rotor(const mppi_model_t* model, float dt, int32_t N, int32_t B, const float* d_x0,
                              const float* d_T0, const float* d_U, float* d_X, float* d_T, void* stream) {
  if (!model || N < 1 || B < 0 || (B > 0 && (!d_x0 || !d_T0 || !d_U || !d_X || !d_T)))
    return fail(MPPI_ERR_ARG, "bad arguments");
  if (model->kind != MPPI_MODEL_ROTOR_RATE) return fail(MPPI_ERR_ARG, "not a rotor model");
  return rollout_states_impl(model, dt, N, B, d_x0, d_U, d_X, stream, d_T0, d_T);
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
static int batch_enqueue(mppi_batch b, const LaunchIO& io, cudaStream_t s);

// Captured form: every rollout group gets its own branch (its own noise
// launch, then its rollout launch), so the groups' kernels overlap and fill
// each other's tails.  The nominal rollouts run at the end of the branch that
// holds every gate-progress solve when there is one such branch, else after
// the branches join.
static int batch_enqueue_branches(mppi_batch b, const LaunchIO& io, cudaStream_t s) {
  const int G = (int)b->rollout_groups.size();
  if (G <= 1 || (int)b->branch_streams.size() < G) return batch_enqueue(b, io, s);
  CU(cudaEventRecord(b->fork, s));
  for (int i = 0; i < G; ++i) {
    const auto& g = b->rollout_groups[i];
    cudaStream_t bs = b->branch_streams[i];
    CU(cudaStreamWaitEvent(bs, b->fork, 0));
    if (g.gen == MPPI_NOISEGEN_KERNEL)
      CU(launch_noise(b->d_descs, g.d_noise_tiles, g.n_tiles, g.block, g.bf16, bs, g.nom, kMaxN));
    CU(launch_rollout(g.objective, g.bf16, b->d_descs, g.d_tiles, g.n_tiles, g.block, g.smem, io, bs, g.gen, g.rot));
    if (i == b->nominal_branch) CU(launch_nominal(b->d_descs, b->d_which, b->n_which, bs));
    CU(cudaEventRecord(b->join[i], bs));
    CU(cudaStreamWaitEvent(s, b->join[i], 0));
  }
  return MPPI_OK;
}

// Captures the plan's launch sequence reading x0 / t0 from and writing u0 to
// the given device buffers (no host-mapped status) and instantiates it.
static int capture_dev_graph(mppi_batch b, const float* x0, const double* t0, float* u0, cudaGraph_t* g,
                             cudaGraphExec_t* e) {
  LaunchIO iod;
  memset(&iod, 0, sizeof iod);
  iod.x0 = x0;
  iod.t0 = t0;
  iod.u0 = u0;
  iod.status = nullptr;
  if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(MPPI_ERR_CUDA, "begin capture failed");
  const int rc = batch_enqueue_branches(b, iod, b->cap_stream);
  const cudaError_t e2 =
      b->nominal_branch < 0 ? launch_nominal(b->d_descs, b->d_which, b->n_which, b->cap_stream) : cudaSuccess;
  cudaGraph_t graph = nullptr;
  const cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &graph);
  if (rc || e2 != cudaSuccess || e3 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(MPPI_ERR_CUDA, "graph capture failed");
  }
  if (cudaGraphInstantiate(e, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(MPPI_ERR_CUDA, "graph instantiation failed");
  }
  *g = graph;
  return MPPI_OK;
}

static int batch_enqueue(mppi_batch b, const LaunchIO& io, cudaStream_t s) {
  for (const auto& g : b->noise_groups)
    CU(launch_noise(b->d_descs, g.d_tiles, g.n_tiles, g.block, g.bf16, s, g.nom, kMaxN));
  for (const auto& g : b->rollout_groups)
    CU(launch_rollout(g.objective, g.bf16, b->d_descs, g.d_tiles, g.n_tiles, g.block, g.smem, io, s, g.gen, g.rot));
  return MPPI_OK;
}

int mppi_batch_destroy(mppi_batch b) {
  if (!b) return MPPI_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->exec_dev) cudaGraphExecDestroy(b->exec_dev);
  if (b->graph_dev) cudaGraphDestroy(b->graph_dev);
  for (const auto& de : b->dev_execs) {
    cudaGraphExecDestroy(de.exec);
    cudaGraphDestroy(de.graph);
  }
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaStream_t bs : b->branch_streams) cudaStreamDestroy(bs);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->ev) cudaEventDestroy(b->ev);
  hostio_free(b->io);
  if (b->dev) cudaFree(b->dev);
  delete b;
  return MPPI_OK;
}

int mppi_batch_create(int32_t n, const mppi_handle* hs, int32_t use_graph, mppi_batch* out) {
  if (!out || n < 1 || !hs) return fail(MPPI_ERR_ARG, "bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return fail(MPPI_ERR_ARG, "null handle at %d", i);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (hs[i] == hs[j]) return fail(MPPI_ERR_ARG, "handle %d appears twice in the batch", i);
  mppi_batch b = new mppi_batch_s();
  b->n = n;
  b->hs.assign(hs, hs + n);
  for (int i = 0; i < n; ++i) b->versions.push_back(hs[i]->version);
  b->use_graph = use_graph != 0;
  b->branches = use_graph == 1;
  // group tiles by launch configuration; longest horizons first (LPT)
  struct Key {
    int obj, bf16, block, gen, nom, rot;
    bool operator<(const Key& o) const {
      if (obj != o.obj) return obj < o.obj;
      if (bf16 != o.bf16) return bf16 < o.bf16;
      if (block != o.block) return block < o.block;
      if (gen != o.gen) return gen < o.gen;
      if (nom != o.nom) return nom < o.nom;
      return rot < o.rot;
    }
  };
  std::vector<std::pair<Key, std::vector<Tile>>> rg;
  std::vector<std::pair<Key, std::vector<Tile>>> ng;
  std::vector<uint32_t> rsmem;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  // longest tiles first: a tile's time grows with N (it holds <= block samples)
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    if (hs[a]->hd.N != hs[c]->hd.N) return hs[a]->hd.N > hs[c]->hd.N;
    return hs[a]->hd.K > hs[c]->hd.K;
  });
  std::vector<int32_t> which;
  for (int oi = 0; oi < n; ++oi) {
    const int i = order[oi];
    const SolveDesc& d = hs[i]->hd;
    // a batch draws the normals of noise-ahead handles before the rollout,
    // as for the separate pass
    const int gen = d.noise_gen == MPPI_NOISEGEN_AHEAD ? MPPI_NOISEGEN_KERNEL : d.noise_gen;
    Key k{d.objective, d.noise_bf16, d.block, gen, d.nominal_sample, d.rotor};
    Key kn{0, d.noise_bf16, d.block, 0, d.nominal_sample, 0};
    auto find = [](std::vector<std::pair<Key, std::vector<Tile>>>& v, const Key& key) -> int {
      for (size_t j = 0; j < v.size(); ++j)
        if (!(v[j].first < key) && !(key < v[j].first)) return (int)j;
      v.push_back({key, {}});
      return (int)v.size() - 1;
    };
    int gi = find(rg, k);
    if ((int)rsmem.size() < (int)rg.size()) rsmem.push_back(0);
    rsmem[gi] =
        std::max(rsmem[gi], rollout_smem_bytes(d.N, d.objective, d.S, tile_samples(d), merge_cap(d.n_tiles),
                                               gen, d.ref_rows));
    const int gn = gen != MPPI_NOISEGEN_KERNEL ? -1 : find(ng, kn);
    for (int t = 0; t < d.n_tiles; ++t) {
      rg[gi].second.push_back(Tile{i, t * tile_samples(d)});
      if (gn >= 0) ng[gn].second.push_back(Tile{i, t * tile_samples(d)});
    }
    if (d.objective == MPPI_OBJ_GATE) which.push_back(i);
  }
  size_t tiles_total = 0;
  for (auto& g : rg) tiles_total += g.second.size();
  for (auto& g : ng) tiles_total += g.second.size();
  const size_t bytes = al256(sizeof(SolveDesc) * n) + al256(sizeof(Tile) * tiles_total) +
                       al256(sizeof(int32_t) * (which.size() + 1)) + al256(sizeof(float) * 13 * n) +
                       al256(sizeof(double) * n) + al256(sizeof(float) * 5 * n);
  if (cudaMalloc(&b->dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(MPPI_ERR_OOM, "batch allocation failed");
  }
  char* c = static_cast<char*>(b->dev);
  b->d_descs = reinterpret_cast<SolveDesc*>(c);
  std::vector<SolveDesc> descs(n);
  for (int i = 0; i < n; ++i) descs[i] = hs[i]->hd;
  auto cleanup = [&](int code) {
    mppi_batch_destroy(b);
    return code;
  };
  if (cudaMemcpy(b->d_descs, descs.data(), sizeof(SolveDesc) * n, cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "descriptor upload failed"));
  c += al256(sizeof(SolveDesc) * n);
  Tile* tp = reinterpret_cast<Tile*>(c);
  for (size_t gi = 0; gi < rg.size(); ++gi) {
    auto& v = rg[gi].second;
    if (cudaMemcpy(tp, v.data(), sizeof(Tile) * v.size(), cudaMemcpyHostToDevice))
      return cleanup(fail(MPPI_ERR_CUDA, "tile upload failed"));
    const Key& k = rg[gi].first;
    b->rollout_groups.push_back({k.obj, k.bf16, k.block, k.gen, k.nom, k.rot, rsmem[gi], (int)v.size(), tp, tp});
    tp += v.size();
  }
  for (auto& g : ng) {
    auto& v = g.second;
    if (cudaMemcpy(tp, v.data(), sizeof(Tile) * v.size(), cudaMemcpyHostToDevice))
      return cleanup(fail(MPPI_ERR_CUDA, "tile upload failed"));
    b->noise_groups.push_back({g.first.bf16, g.first.block, g.first.nom, (int)v.size(), tp});
    tp += v.size();
  }
  c += al256(sizeof(Tile) * tiles_total);
  b->d_which = reinterpret_cast<int32_t*>(c);
  c += al256(sizeof(int32_t) * (which.size() + 1));
  b->d_x0s = reinterpret_cast<float*>(c);
  c += al256(sizeof(float) * 13 * n);
  b->d_t0s = reinterpret_cast<double*>(c);
  c += al256(sizeof(double) * n);
  b->d_u0s = reinterpret_cast<float*>(c);
  b->n_which = (int)which.size();
  if (!which.empty() && cudaMemcpy(b->d_which, which.data(), sizeof(int32_t) * which.size(), cudaMemcpyHostToDevice))
    return cleanup(fail(MPPI_ERR_CUDA, "work list upload failed"));
  b->kernels_per_solve = (int)b->noise_groups.size() + (int)b->rollout_groups.size() + (b->n_which > 0 ? 1 : 0);
  if (b->use_graph && b->branches && b->rollout_groups.size() > 1 && b->rollout_groups.size() <= 8) {
    b->kernels_per_solve = b->n_which > 0 ? 1 : 0;
    for (const auto& g : b->rollout_groups) b->kernels_per_solve += g.gen == MPPI_NOISEGEN_KERNEL ? 2 : 1;
  }
  int rc = hostio_alloc(b->io, n);
  if (rc) return cleanup(rc);
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(MPPI_ERR_CUDA, "event creation failed"));
  if (b->use_graph) {
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(MPPI_ERR_CUDA, "stream creation failed"));
    const int G = (int)b->rollout_groups.size();
    if (b->branches && G > 1 && G <= 8) {
      if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(MPPI_ERR_CUDA, "event creation failed"));
      for (int i = 0; i < G; ++i) {
        cudaStream_t bs;
        if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess)
          return cleanup(fail(MPPI_ERR_CUDA, "stream creation failed"));
        b->branch_streams.push_back(bs);
        if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
          return cleanup(fail(MPPI_ERR_CUDA, "event creation failed"));
      }
      int gate_groups = 0, gate_at = -1;
      for (int i = 0; i < G; ++i)
        if (b->rollout_groups[i].objective == MPPI_OBJ_GATE) {
          ++gate_groups;
          gate_at = i;
        }
      if (gate_groups == 1 && b->n_which > 0) b->nominal_branch = gate_at;
    }
    LaunchIO io;
    memset(&io, 0, sizeof io);
    io.x0 = b->io.d_x0;
    io.t0 = b->io.d_t0;
    io.u0 = b->io.d_u0;
    io.status = b->io.d_status;
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return cleanup(fail(MPPI_ERR_CUDA, "begin capture failed"));
    int rc2 = batch_enqueue_branches(b, io, b->cap_stream);
    cudaError_t e1 = cudaEventRecordWithFlags(b->ev, b->cap_stream, cudaEventRecordExternal);
    cudaError_t e2 =
        b->nominal_branch < 0 ? launch_nominal(b->d_descs, b->d_which, b->n_which, b->cap_stream) : cudaSuccess;
    cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (rc2 || e1 || e2 || e3)
      return cleanup(fail(MPPI_ERR_CUDA, "graph capture failed (%s / %s / %s)", cudaGetErrorString(e1),
                          cudaGetErrorString(e2), cudaGetErrorString(e3)));
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
      return cleanup(fail(MPPI_ERR_CUDA, "graph instantiation failed"));
    int rc3 = capture_dev_graph(b, b->d_x0s, b->d_t0s, b->d_u0s, &b->graph_dev, &b->exec_dev);
    if (rc3) return cleanup(rc3);
  }
  *out = b;
  return MPPI_OK;
}

static int batch_check(mppi_batch b, cudaStream_t s) {
  for (int i = 0; i < b->n; ++i)
    if (b->hs[i]->version != b->versions[i]) return fail(MPPI_ERR_ARG, "handle %d changed shape since the batch was planned", i);
  for (int i = 0; i < b->n; ++i)
    if (b->hs[i]->ext_noise_pending) return fail(MPPI_ERR_ARG, "caller noise is only supported for single solves");
  // the batch draws its own normals and moves every counter on: what a
  // noise-ahead handle drew after its last single solve is stale after it.
  // That draw may still run on another stream: the batch waits for it.
  for (int i = 0; i < b->n; ++i) {
    const int rc = wait_ahead(b->hs[i], s);
    if (rc) return rc;
    b->hs[i]->ahead_ready = false;
  }
  return MPPI_OK;
}

int mppi_batch_solve(mppi_batch b, const float* x0s, const double* t0s, void* stream, float* u0s_out) {
  if (!b || !x0s || !u0s_out) return fail(MPPI_ERR_ARG, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = batch_check(b, s);
  if (rc) return rc;
  memcpy(b->io.x0, x0s, sizeof(float) * 13 * b->n);
  if (t0s)
    memcpy(b->io.t0, t0s, sizeof(double) * b->n);
  else
    memset(b->io.t0, 0, sizeof(double) * b->n);
  if (b->use_graph) {
    CU(cudaGraphLaunch(b->exec, s));
    add_launches(b->kernels_per_solve);
  } else {
    LaunchIO io;
    memset(&io, 0, sizeof io);
    io.x0 = b->io.d_x0;
    io.t0 = b->io.d_t0;
    io.u0 = b->io.d_u0;
    io.status = b->io.d_status;
    rc = batch_enqueue(b, io, s);
    if (rc) return rc;
    CU(cudaEventRecord(b->ev, s));
    CU(launch_nominal(b->d_descs, b->d_which, b->n_which, s));
  }
  CU(cudaEventSynchronize(b->ev));
  memcpy(u0s_out, (const void*)b->io.u0, sizeof(float) * 5 * b->n);
  for (int i = 0; i < b->n; ++i)
    if (((volatile int32_t*)b->io.status)[i] == MPPI_ERR_TIMEOUT)
      return fail(MPPI_ERR_TIMEOUT, "solve %d: a bounded wait for the bulk copies gave up", i);
  for (int i = 0; i < b->n; ++i)
    if (((volatile int32_t*)b->io.status)[i] == MPPI_WARN_DEGENERATE)
      return fail(MPPI_WARN_DEGENERATE, "solve %d: every sample cost was non-finite", i);
  return MPPI_OK;
}

int mppi_batch_profile(mppi_batch b, int32_t n_iters, void* stream, float ms_out[6]) {
  if (!b || n_iters < 1 || !ms_out) return fail(MPPI_ERR_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = batch_check(b, s);
  if (rc) return rc;
  LaunchIO io;
  memset(&io, 0, sizeof io);
  io.x0 = b->io.d_x0;
  io.t0 = b->io.d_t0;
  io.u0 = b->io.d_u0;
  io.status = b->io.d_status;
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) CU(cudaEventCreate(&ev[i]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  int status = MPPI_OK;
  for (int it = 0; it < n_iters && status == MPPI_OK; ++it) {
    cudaEventRecord(ev[0], s);
    for (const auto& g : b->noise_groups)
      if (launch_noise(b->d_descs, g.d_tiles, g.n_tiles, g.block, g.bf16, s, g.nom, kMaxN) != cudaSuccess)
        status = MPPI_ERR_CUDA;
    cudaEventRecord(ev[1], s);
    for (int obj = 0; obj < 3; ++obj) {
      for (const auto& g : b->rollout_groups)
        if (g.objective == obj &&
            launch_rollout(g.objective, g.bf16, b->d_descs, g.d_tiles, g.n_tiles, g.block, g.smem, io, s, g.gen,
                           g.rot) !=
                cudaSuccess)
          status = MPPI_ERR_CUDA;
      cudaEventRecord(ev[2 + obj], s);
    }
    if (launch_nominal(b->d_descs, b->d_which, b->n_which, s) != cudaSuccess) status = MPPI_ERR_CUDA;
    cudaEventRecord(ev[5], s);
    if (cudaEventSynchronize(ev[5]) != cudaSuccess) status = MPPI_ERR_CUDA;
    float t;
    cudaEventElapsedTime(&t, ev[0], ev[1]); acc[0] += t;
    cudaEventElapsedTime(&t, ev[1], ev[2]); acc[1] += t;
    cudaEventElapsedTime(&t, ev[2], ev[3]); acc[2] += t;
    cudaEventElapsedTime(&t, ev[3], ev[4]); acc[3] += t;
    cudaEventElapsedTime(&t, ev[4], ev[5]); acc[4] += t;
    cudaEventElapsedTime(&t, ev[0], ev[5]); acc[5] += t;
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  if (status) return fail(status, "profiled launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  for (int i = 0; i < 6; ++i) ms_out[i] = (float)(acc[i] / n_iters);
  return MPPI_OK;
}

int mppi_batch_solve_async(mppi_batch b, const float* d_x0s, const double* d_t0s, void* stream, float* d_u0s) {
  if (!b || !d_x0s || !d_u0s) return fail(MPPI_ERR_ARG, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = batch_check(b, s);
  if (rc) return rc;
  LaunchIO io;
  memset(&io, 0, sizeof io);
  io.x0 = d_x0s;
  io.t0 = d_t0s;
  io.u0 = d_u0s;
  io.status = nullptr;
  if (!d_t0s) return fail(MPPI_ERR_ARG, "d_t0s is required");
  if (b->use_graph && b->exec_dev) {
    // the caller's buffers directly, through a graph captured on them
    cudaGraphExec_t ex = nullptr;
    for (const auto& de : b->dev_execs)
      if (de.x0 == d_x0s && de.t0 == d_t0s && de.u0 == d_u0s) ex = de.exec;
    if (!ex && b->dev_execs.size() < kMaxDevExecs) {
      mppi_batch_s::DevExec de{d_x0s, d_t0s, d_u0s, nullptr, nullptr};
      rc = capture_dev_graph(b, d_x0s, d_t0s, d_u0s, &de.graph, &de.exec);
      if (rc) return rc;
      b->dev_execs.push_back(de);
      ex = de.exec;
    }
    if (ex) {
      CU(cudaGraphLaunch(ex, s));
      add_launches(b->kernels_per_solve);
      return MPPI_OK;
    }
    // more pointer sets than kept graphs: copy through the plan's own buffers
    CU(cudaMemcpyAsync(b->d_x0s, d_x0s, sizeof(float) * 13 * b->n, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(b->d_t0s, d_t0s, sizeof(double) * b->n, cudaMemcpyDeviceToDevice, s));
    CU(cudaGraphLaunch(b->exec_dev, s));
    add_launches(b->kernels_per_solve);
    CU(cudaMemcpyAsync(d_u0s, b->d_u0s, sizeof(float) * 5 * b->n, cudaMemcpyDeviceToDevice, s));
    return MPPI_OK;
  }
  rc = batch_enqueue(b, io, s);
  if (rc) return rc;
  CU(launch_nominal(b->d_descs, b->d_which, b->n_which, s));
  return MPPI_OK;
}

// mppi_solve_batch: cached plans keyed by the handle list (g_plans)

int mppi_solve_batch(int32_t n, const mppi_handle* hs, const float* x0s, const double* t0s, void* stream,
                     float* u0s_out) {
  if (n < 1 || !hs || !x0s || !u0s_out) return fail(MPPI_ERR_ARG, "bad arguments");
  mppi_batch plan = nullptr;
  // a plan leaves the cache when it goes stale, when the cache is full or
  // when one of its handles is destroyed; one that a call is running is only
  // marked, and its last user destroys it
  auto drop = [](mppi_batch p) {
    if (p->users == 0)
      mppi_batch_destroy(p);
    else
      p->evicted = true;
  };
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (size_t i = 0; i < g_plans.size(); ++i) {
      mppi_batch p = g_plans[i];
      if (p->n != n || !std::equal(p->hs.begin(), p->hs.end(), hs)) continue;
      bool fresh = true;
      for (int j = 0; j < n; ++j) fresh = fresh && p->versions[j] == hs[j]->version;
      if (fresh) {
        plan = p;
      } else {
        g_plans.erase(g_plans.begin() + i);
        drop(p);
      }
      break;
    }
    if (!plan) {
      int rc = mppi_batch_create(n, hs, 1, &plan);
      if (rc) return rc;
      if (g_plans.size() >= 8) {
        mppi_batch old = g_plans.front();
        g_plans.erase(g_plans.begin());
        drop(old);
      }
      g_plans.push_back(plan);
    }
    ++plan->users;
  }
  const int rc = mppi_batch_solve(plan, x0s, t0s, stream, u0s_out);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (--plan->users == 0 && plan->evicted) mppi_batch_destroy(plan);
  }
  return rc;
}

}  // extern "C"
