// mppi_serve.cu -- continuous batching of many drones' MPPI solves.
//
// Every drone keeps only its resident controller state on the device (the
// nominal U*, Philox iteration, gate index, pass counts of the previous
// nominal, progress state, merge tickets, track tables).  The per-solve
// scratch (standard normals, per-sample costs, tile partials) belongs to a
// request and is carved from one device pool of a fixed budget when the
// request is admitted; it returns to the pool when the request finishes.
// Admission is first-come first-served: the queue head is admitted when its
// drone is idle and its scratch fits in the pool (requests of busy drones are
// passed over, a request that does not fit stops the batch).  A batch runs
// the same kernels as mppi_solve_batch on one of several streams, so batches
// overlap on the device while later requests are queued.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "mppi_device.cuh"
#include "mppi_launch.h"

using namespace mppi;

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int sfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define SCU(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return sfail(MPPI_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over the device pool (host bookkeeping only).
class Pool {
 public:
  void reset(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    size_ = bytes;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

struct Drone {
  mppi_model_t model;
  mppi_params_t params;
  int nu = 4, block = 128, K_cap = 0, N_cap = 0;
  void* slab = nullptr;  // resident state + tables + tickets
  SolveDesc hd;          // template: resident pointers filled, scratch pointers per request
  bool busy = false;
};

struct Request {
  int64_t id;
  int32_t drone;
  float x0[kNX];
  double t0;
  int32_t K, N;
  double t_submit, t_launch;
  double deadline = 0.0;      // mppi_clock() after which it is not launched (0: none)
  size_t off = 0, bytes = 0;  // scratch in the pool
};

// scratch bytes of one request and the offsets of its parts
struct Scratch {
  size_t Z, Z5, J, info, pm, pS, pP, total;
};

Scratch scratch_for(int K, int N, int block, int five, int bf16, int gen) {
  const int T = (K + block - 1) / block;
  int sq = 1;
  while (sq * sq < T) ++sq;
  const int Gn = 2 * sq + 16;
  Scratch s;
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o = al256(o + b);
    return r;
  };
  // regenerated noise and noise kept in shared memory need no buffer
  const bool stored = gen != MPPI_NOISEGEN_REGEN && gen != MPPI_NOISEGEN_SMEM;
  s.Z = take(stored ? (size_t)N * K * (bf16 ? 8 : 16) : 16);
  s.Z5 = take(five && stored ? (size_t)N * K * (bf16 ? 2 : 4) : 16);
  s.J = take(sizeof(double) * K);
  s.info = take(sizeof(int32_t) * K);
  s.pm = take(sizeof(double) * (T + Gn + 1));
  s.pS = take(sizeof(double) * (T + Gn + 1));
  s.pP = take(sizeof(double) * (size_t)(T + Gn + 1) * N * kNU);
  s.total = o;
  return s;
}

// one stream slot: a batch in flight and its staging buffers
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request> reqs;
  // pinned, mapped staging: descriptors, tiles, which, x0, t0 (copied to the
  // device in one transfer) and u0 / status (written by the device directly)
  char* host = nullptr;
  char* dev = nullptr;
  float* u0 = nullptr;       // mapped host
  int32_t* status = nullptr;  // mapped host
  float* d_u0 = nullptr;
  int32_t* d_status = nullptr;
  size_t staged_bytes = 0;
};

}  // namespace

struct mppi_server_s {
  int device = 0;
  int max_drones = 0, max_batch = 0, max_tiles = 0;
  double refused = 0.0;  // requests dropped past their deadline
  bool fail_next_launch = false;  // testing hook: the next admitted batch fails on the host
  std::vector<Drone> drones;
  char* pool_base = nullptr;
  Pool pool;
  std::deque<Request> queue;
  std::vector<Slot> slots;
  int next_slot = 0;
  int64_t next_id = 1;
  double batches = 0, finished = 0;
  std::vector<mppi_result_t> done;  // finished, not yet polled
  std::mutex mu;
};

namespace {

// staging layout of a slot (offsets into host / dev buffers)
struct Staging {
  size_t descs, tiles, which, x0, t0, total;
};

Staging staging_for(int max_batch, int max_tiles) {
  Staging st;
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o = al256(o + b);
    return r;
  };
  st.descs = take(sizeof(SolveDesc) * max_batch);
  st.tiles = take(sizeof(Tile) * (size_t)max_tiles);
  st.which = take(sizeof(int32_t) * (max_batch + 1));
  st.x0 = take(sizeof(float) * kNX * max_batch);
  st.t0 = take(sizeof(double) * max_batch);
  st.total = o;
  return st;
}

void destroy_server(mppi_server s) {
  for (auto& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.dev) cudaFree(sl.dev);
    if (sl.u0) cudaFreeHost(sl.u0);
  }
  for (auto& d : s->drones)
    if (d.slab) cudaFree(d.slab);
  if (s->pool_base) cudaFree(s->pool_base);
  delete s;
}

}  // namespace

extern "C" {

double mppi_clock(void) { return now_s(); }

int mppi_server_create(int32_t max_drones, size_t scratch_budget_bytes, int32_t n_slots, int32_t max_batch,
                       mppi_server* out) {
  if (!out || max_drones < 1 || n_slots < 1 || n_slots > 16 || max_batch < 1 || scratch_budget_bytes < 4096)
    return sfail(MPPI_ERR_ARG, "mppi_server_create: bad arguments");
  *out = nullptr;
  mppi_server s = new mppi_server_s();
  s->max_drones = max_drones;
  s->max_batch = max_batch;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return sfail(MPPI_ERR_CUDA, "mppi_server_create: no device");
  }
  if (configure_kernels() != cudaSuccess) {
    delete s;
    return sfail(MPPI_ERR_CUDA, "mppi_server_create: kernel configuration failed");
  }
  // worst case tiles: every request at the largest K a drone may ask for is
  // not known yet; size for max_batch requests of up to 16384 samples at
  // 32-sample blocks, capped, and check at admission
  s->max_tiles = std::min(max_batch * 512, 1 << 20);
  if (cudaMalloc(&s->pool_base, scratch_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return sfail(MPPI_ERR_OOM, "mppi_server_create: pool of %zu bytes", scratch_budget_bytes);
  }
  s->pool.reset(scratch_budget_bytes);
  const Staging st = staging_for(max_batch, s->max_tiles);
  s->slots.resize(n_slots);
  for (auto& sl : s->slots) {
    void* h = nullptr;
    void* u = nullptr;
    const size_t ub = al256(sizeof(float) * kNU * max_batch) + al256(sizeof(int32_t) * max_batch);
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc(&h, st.total, cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&sl.dev), st.total) != cudaSuccess ||
        cudaHostAlloc(&u, ub, cudaHostAllocMapped) != cudaSuccess) {
      sl.host = static_cast<char*>(h);
      sl.u0 = static_cast<float*>(u);
      cudaGetLastError();
      destroy_server(s);
      return sfail(MPPI_ERR_OOM, "mppi_server_create: slot buffers");
    }
    sl.host = static_cast<char*>(h);
    sl.u0 = static_cast<float*>(u);
    sl.status = reinterpret_cast<int32_t*>(static_cast<char*>(u) + al256(sizeof(float) * kNU * max_batch));
    void* du = nullptr;
    if (cudaHostGetDevicePointer(&du, u, 0) != cudaSuccess) {
      destroy_server(s);
      return sfail(MPPI_ERR_CUDA, "mppi_server_create: mapped pointer");
    }
    sl.d_u0 = static_cast<float*>(du);
    sl.d_status = reinterpret_cast<int32_t*>(static_cast<char*>(du) + al256(sizeof(float) * kNU * max_batch));
  }
  s->drones.reserve(max_drones);
  *out = s;
  return MPPI_OK;
}

int mppi_server_add_drone(mppi_server s, const mppi_model_t* model, const mppi_params_t* params,
                          const mppi_track_t* track, int32_t* drone_out) {
  if (!s || !model || !params || !track || !drone_out) return sfail(MPPI_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->drones.size() >= s->max_drones) return sfail(MPPI_ERR_NOT_ADMITTED, "server holds max_drones drones");
  if (model->kind != MPPI_MODEL_CTBR && model->kind != MPPI_MODEL_ROTOR_RATE) return sfail(MPPI_ERR_ARG, "model kind");
  if (model->kind == MPPI_MODEL_ROTOR_RATE &&
      (params->noise_dtype != MPPI_NOISE_F32 || !(model->arm > 0) || !(model->thrust_max > model->thrust_min)))
    return sfail(MPPI_ERR_ARG, "rotor model: float32 noise, arm > 0, thrust_max > thrust_min");
  const mppi_params_t& p = *params;
  const int block = p.block ? p.block : 128;
  if (block < 32 || block > std::min(128, rollout_max_block()) || block % 32)
    return sfail(MPPI_ERR_ARG, "server drones use blocks of 32..128 threads");
  const int K_cap = p.K_cap ? p.K_cap : p.K, N_cap = p.N_cap ? p.N_cap : p.N;
  if (p.K < 1 || p.N < 1 || K_cap < p.K || N_cap < p.N || N_cap > MPPI_MAX_N)
    return sfail(MPPI_ERR_ARG, "bad K / N caps");
  if ((K_cap + block - 1) / block > s->max_tiles) return sfail(MPPI_ERR_ARG, "K_cap too large for this server");
  if (p.objective < 0 || p.objective > 2) return sfail(MPPI_ERR_ARG, "unknown objective");
  if (p.noise_dtype != MPPI_NOISE_F32 && p.noise_dtype != MPPI_NOISE_BF16) return sfail(MPPI_ERR_ARG, "noise dtype");
  if (p.accum < 0 || p.accum > 2) return sfail(MPPI_ERR_ARG, "unknown accumulation mode");
  if (p.noise_gen == MPPI_NOISEGEN_AHEAD)
    return sfail(MPPI_ERR_ARG, "noise drawn ahead is for single solves: a served drone draws its own");
  if (p.noise_gen < MPPI_NOISEGEN_KERNEL || p.noise_gen > MPPI_NOISEGEN_SMEM ||
      (p.noise_gen == MPPI_NOISEGEN_REGEN && p.noise_dtype != MPPI_NOISE_F32))
    return sfail(MPPI_ERR_ARG, "bad noise generation mode");
  if (p.noise_gen == MPPI_NOISEGEN_SMEM) {
    const int tile = block * (p.samples_per_thread ? p.samples_per_thread : 1);
    const int rows = p.objective == MPPI_OBJ_TRACK ? ref_rows_for(N_cap, p.dt, track->dt_ref, track->T) : 0;
    if (rollout_smem_bytes(N_cap, p.objective, track->S, tile, std::max(32, (K_cap + tile - 1) / tile),
                           MPPI_NOISEGEN_SMEM, rows) > kRolloutSmemMax)
      return sfail(MPPI_ERR_ARG, "noise kept in shared memory does not fit a block's shared memory");
  }
  if (p.samples_per_thread < 0 || p.samples_per_thread > MPPI_MAX_SPT)
    return sfail(MPPI_ERR_ARG, "samples_per_thread outside [0, %d]", MPPI_MAX_SPT);
  if (track->n_gates < 0 || track->n_gates > MPPI_MAX_GATES) return sfail(MPPI_ERR_ARG, "n_gates out of range");
  if (p.objective == MPPI_OBJ_GATE && (track->n_gates < 1 || !track->gates)) return sfail(MPPI_ERR_ARG, "no gates");
  if (p.objective == MPPI_OBJ_CONTOUR && (track->S < 2 || !track->path || !(track->L > 0)))
    return sfail(MPPI_ERR_ARG, "contouring needs a path table");
  if (p.objective == MPPI_OBJ_TRACK && (track->T < 2 || !track->ref || !(track->dt_ref > 0)))
    return sfail(MPPI_ERR_ARG, "tracking needs a reference table");
  Drone d;
  d.model = *model;
  d.params = p;
  d.params.block = block;
  d.block = block;
  d.K_cap = K_cap;
  d.N_cap = N_cap;
  d.nu = p.objective == MPPI_OBJ_CONTOUR ? 5 : 4;
  const int T_cap = (K_cap + block - 1) / block;
  int sq = 1;
  while (sq * sq < T_cap) ++sq;
  const int Gn = 2 * sq + 16;
  // resident slab
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o = al256(o + b);
    return r;
  };
  const size_t o_st = take(sizeof(DevState)), o_U = take(sizeof(float) * (N_cap * kNU + 8)),
               o_prev = take(sizeof(int32_t) * (N_cap + 8)), o_g = take(sizeof(float) * 6 * std::max(1, track->n_gates)),
               o_gf = take(sizeof(GateF) * std::max(1, track->n_gates)),
               o_path = take(sizeof(float) * 6 * std::max(1, track->S) + 64),
               o_ref = take(sizeof(float) * 13 * std::max(1, track->T) + 64), o_unew = take(sizeof(float) * N_cap * kNU),
               o_pc = take(sizeof(int32_t) * (N_cap + 1)), o_xref = take(sizeof(float) * 13 * (N_cap + 1)),
               o_tk = take(sizeof(uint32_t) * (Gn + 2));
  if (cudaMalloc(&d.slab, o) != cudaSuccess) {
    cudaGetLastError();
    return sfail(MPPI_ERR_OOM, "drone state of %zu bytes", o);
  }
  char* b = static_cast<char*>(d.slab);
  SCU(cudaMemset(d.slab, 0, o));
  memset(&d.hd, 0, sizeof d.hd);
  fill_model_params(d.model, d.params, d.nu, d.hd);
  SolveDesc& h = d.hd;
  h.st = reinterpret_cast<DevState*>(b + o_st);
  h.U = reinterpret_cast<float*>(b + o_U);
  h.prevcnt = reinterpret_cast<int32_t*>(b + o_prev);
  h.N_cap = N_cap;
  h.gates = reinterpret_cast<float*>(b + o_g);
  h.n_gates = track->n_gates;
  h.closed = track->closed ? 1 : 0;
  h.path = reinterpret_cast<float*>(b + o_path);
  h.S = track->S;
  h.L = track->L;
  h.ds = track->S > 0 ? (float)((double)track->L / track->S) : 1.f;
  h.inv_ds = track->S > 0 ? (float)((double)track->S / track->L) : 1.f;
  h.ref = reinterpret_cast<float*>(b + o_ref);
  h.T = track->T;
  h.dt_ref = track->dt_ref;
  h.gframes = reinterpret_cast<const GateF*>(b + o_gf);
  h.ref_rows = p.objective == MPPI_OBJ_TRACK ? ref_rows_for(N_cap, p.dt, track->dt_ref, track->T) : 0;
  h.ref_pad = 64;
  h.unew = reinterpret_cast<float*>(b + o_unew);
  h.passcnt = reinterpret_cast<int32_t*>(b + o_pc);
  h.xref = reinterpret_cast<float*>(b + o_xref);
  h.ticket = reinterpret_cast<uint32_t*>(b + o_tk);
  h.block = block;
  if (track->n_gates > 0 && track->gates) {
    SCU(cudaMemcpy((void*)h.gates, track->gates, sizeof(float) * 6 * track->n_gates, cudaMemcpyHostToDevice));
    SCU(launch_gate_frames(h.gates, track->n_gates, const_cast<GateF*>(h.gframes), 0));
    SCU(cudaStreamSynchronize(0));
  }
  if (track->S > 0 && track->path)
    SCU(cudaMemcpy((void*)h.path, track->path, sizeof(float) * 6 * track->S, cudaMemcpyHostToDevice));
  if (track->T > 0 && track->ref)
    SCU(cudaMemcpy((void*)h.ref, track->ref, sizeof(float) * 13 * track->T, cudaMemcpyHostToDevice));
  std::vector<float> U((size_t)N_cap * kNU + 8, 0.f);
  if (model->kind != MPPI_MODEL_ROTOR_RATE)  // hover thrust; the rotor model starts at zero rates
    for (int k = 0; k < N_cap; ++k) U[(size_t)k * kNU] = model->mass * model->gravity;
  SCU(cudaMemcpy(h.U, U.data(), sizeof(float) * U.size(), cudaMemcpyHostToDevice));
  DevState st;
  memset(&st, 0, sizeof st);
  st.c_last = model->mass * model->gravity;
  SCU(cudaMemcpy(h.st, &st, sizeof st, cudaMemcpyHostToDevice));
  *drone_out = (int32_t)s->drones.size();
  s->drones.push_back(d);
  return MPPI_OK;
}

}  // extern "C"

extern "C" {

int mppi_server_submit(mppi_server s, int32_t n, const int32_t* drones, const float* x0s, const double* t0s,
                       const int32_t* Ks, const int32_t* Ns, int64_t* ids_out) {
  return mppi_server_submit_deadline(s, n, drones, x0s, t0s, Ks, Ns, nullptr, ids_out);
}

int mppi_server_submit_deadline(mppi_server s, int32_t n, const int32_t* drones, const float* x0s,
                                const double* t0s, const int32_t* Ks, const int32_t* Ns, const double* deadlines,
                                int64_t* ids_out) {
  if (!s || n < 0 || (n > 0 && (!drones || !x0s || !Ks || !Ns))) return sfail(MPPI_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  for (int i = 0; i < n; ++i) {
    if (drones[i] < 0 || drones[i] >= (int)s->drones.size()) return sfail(MPPI_ERR_ARG, "unknown drone %d", drones[i]);
    const Drone& d = s->drones[drones[i]];
    if (Ks[i] < 1 || Ks[i] > d.K_cap || Ns[i] < 1 || Ns[i] > d.N_cap)
      return sfail(MPPI_ERR_NOT_ADMITTED, "request K=%d N=%d outside drone %d caps", Ks[i], Ns[i], drones[i]);
    const Scratch sc = scratch_for(Ks[i], Ns[i], d.block, d.nu == 5, d.hd.noise_bf16, d.hd.noise_gen);
    if (sc.total > s->pool.size())
      return sfail(MPPI_ERR_NOT_ADMITTED, "request needs %zu scratch bytes, the pool has %zu", sc.total, s->pool.size());
    const int T = (Ks[i] + d.block * d.hd.spt - 1) / (d.block * d.hd.spt);
    if (T > s->max_tiles)
      return sfail(MPPI_ERR_NOT_ADMITTED, "request needs %d tiles, a batch holds %d", T, s->max_tiles);
  }
  const double t = now_s();
  for (int i = 0; i < n; ++i) {
    Request r;
    r.id = s->next_id++;
    r.drone = drones[i];
    memcpy(r.x0, x0s + (size_t)kNX * i, sizeof r.x0);
    r.t0 = t0s ? t0s[i] : 0.0;
    r.K = Ks[i];
    r.N = Ns[i];
    r.t_submit = t;
    r.t_launch = 0.0;
    r.deadline = deadlines ? deadlines[i] : 0.0;
    s->queue.push_back(r);
    if (ids_out) ids_out[i] = r.id;
  }
  return MPPI_OK;
}

int mppi_server_step(mppi_server s, int32_t* launched) {
  if (!s) return sfail(MPPI_ERR_ARG, "null server");
  if (launched) *launched = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->queue.empty()) return MPPI_OK;
  int si = -1;
  for (int t = 0; t < (int)s->slots.size(); ++t) {
    const int c = (s->next_slot + t) % (int)s->slots.size();
    if (!s->slots[c].busy) {
      si = c;
      break;
    }
  }
  if (si < 0) return MPPI_OK;
  Slot& sl = s->slots[si];
  // admission: arrival order, idle drones, scratch from the pool
  std::vector<Request> batch;
  std::deque<Request> keep;
  int tiles = 0;
  bool blocked = false;
  const double t_adm = now_s();
  while (!s->queue.empty()) {
    Request r = s->queue.front();
    s->queue.pop_front();
    if (r.deadline > 0.0 && t_adm > r.deadline) {
      // past its deadline before it could be launched: refused, reported by poll
      mppi_result_t res;
      memset(&res, 0, sizeof res);
      res.request = r.id;
      res.drone = r.drone;
      res.status = MPPI_ERR_NOT_ADMITTED;
      res.K = r.K;
      res.N = r.N;
      res.t_submit = r.t_submit;
      res.t_done = t_adm;
      s->done.push_back(res);
      s->refused += 1.0;
      continue;
    }
    Drone& d = s->drones[r.drone];
    const int TS = d.block * d.hd.spt;
    const int T = (r.K + TS - 1) / TS;
    if (blocked || d.busy || (int)batch.size() >= s->max_batch || tiles + T > s->max_tiles) {
      keep.push_back(r);
      continue;
    }
    const Scratch sc = scratch_for(r.K, r.N, d.block, d.nu == 5, d.hd.noise_bf16, d.hd.noise_gen);
    size_t off = 0;
    if (!s->pool.alloc(sc.total, &off)) {
      blocked = true;  // the head waits for memory; later arrivals do not jump it
      keep.push_back(r);
      continue;
    }
    r.off = off;
    r.bytes = sc.total;
    d.busy = true;
    tiles += T;
    batch.push_back(r);
  }
  s->queue.swap(keep);
  if (batch.empty()) return MPPI_OK;

  // descriptors of this batch, pointing at the drones' resident state and at
  // the requests' scratch; the staging area is packed for this batch
  // (descriptors, tiles, gate work list, x0, t0) and sent in one transfer
  const int nb = (int)batch.size();
  Staging st;
  {
    size_t o = 0;
    auto take = [&](size_t b) {
      const size_t r = o;
      o = al256(o + b);
      return r;
    };
    st.descs = take(sizeof(SolveDesc) * nb);
    st.tiles = take(sizeof(Tile) * (size_t)tiles);
    st.which = take(sizeof(int32_t) * (nb + 1));
    st.x0 = take(sizeof(float) * kNX * nb);
    st.t0 = take(sizeof(double) * nb);
    st.total = o;
  }
  SolveDesc* hdesc = reinterpret_cast<SolveDesc*>(sl.host + st.descs);
  float* hx0 = reinterpret_cast<float*>(sl.host + st.x0);
  double* ht0 = reinterpret_cast<double*>(sl.host + st.t0);
  const double tl = now_s();
  for (size_t i = 0; i < batch.size(); ++i) {
    Request& r = batch[i];
    const Drone& d = s->drones[r.drone];
    SolveDesc dd = d.hd;
    char* b = s->pool_base + r.off;
    const Scratch sc = scratch_for(r.K, r.N, d.block, d.nu == 5, dd.noise_bf16, dd.noise_gen);
    dd.K = r.K;
    dd.N = r.N;
    dd.n_tiles = (r.K + tile_samples(dd) - 1) / tile_samples(dd);
    const bool stored = dd.noise_gen != MPPI_NOISEGEN_REGEN && dd.noise_gen != MPPI_NOISEGEN_SMEM;
    dd.Z4 = (stored && !dd.noise_bf16) ? reinterpret_cast<float4*>(b + sc.Z) : nullptr;
    dd.Zb = (stored && dd.noise_bf16) ? reinterpret_cast<uint2*>(b + sc.Z) : nullptr;
    dd.Z5 = (stored && d.nu == 5 && !dd.noise_bf16) ? reinterpret_cast<float*>(b + sc.Z5) : nullptr;
    dd.Z5b = (stored && d.nu == 5 && dd.noise_bf16) ? reinterpret_cast<__nv_bfloat16*>(b + sc.Z5) : nullptr;
    dd.J = reinterpret_cast<double*>(b + sc.J);
    dd.info = reinterpret_cast<int32_t*>(b + sc.info);
    dd.part_m = reinterpret_cast<double*>(b + sc.pm);
    dd.part_S = reinterpret_cast<double*>(b + sc.pS);
    dd.part_P = reinterpret_cast<double*>(b + sc.pP);
    dd.ext_noise = 0;
    hdesc[i] = dd;
    memcpy(hx0 + (size_t)kNX * i, r.x0, sizeof r.x0);
    ht0[i] = r.t0;
    r.t_launch = tl;
  }
  // tiles: rollout groups by (objective, noise type, block), longest
  // horizons first; the noise launches reuse the same tiles per (type, block)
  struct Group {
    int obj, bf16, block, gen, nom, rot;
    std::vector<Tile> t;
    uint32_t smem = 0;
  };
  std::vector<Group> groups;
  std::vector<int> order(batch.size());
  for (size_t i = 0; i < batch.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return batch[a].N > batch[c].N; });
  std::vector<int32_t> which;
  for (int i : order) {
    const SolveDesc& dd = hdesc[i];
    int g = -1;
    for (size_t q = 0; q < groups.size(); ++q)
      if (groups[q].obj == dd.objective && groups[q].bf16 == dd.noise_bf16 && groups[q].block == dd.block &&
          groups[q].gen == dd.noise_gen && groups[q].nom == dd.nominal_sample && groups[q].rot == dd.rotor)
        g = (int)q;
    if (g < 0) {
      groups.push_back(Group{dd.objective, dd.noise_bf16, dd.block, dd.noise_gen, dd.nominal_sample, dd.rotor, {}, 0});
      g = (int)groups.size() - 1;
    }
    for (int t = 0; t < dd.n_tiles; ++t) groups[g].t.push_back(Tile{i, t * tile_samples(dd)});
    groups[g].smem = std::max(groups[g].smem, rollout_smem_bytes(dd.N, dd.objective, dd.S, tile_samples(dd),
                                                                 dd.n_tiles > 32 ? dd.n_tiles : 32, dd.noise_gen,
                                                                 dd.ref_rows));
    if (dd.objective == MPPI_OBJ_GATE) which.push_back(i);
  }
  Tile* htiles = reinterpret_cast<Tile*>(sl.host + st.tiles);
  std::vector<size_t> goff(groups.size());
  size_t nt = 0;
  for (size_t q = 0; q < groups.size(); ++q) {
    goff[q] = nt;
    memcpy(htiles + nt, groups[q].t.data(), sizeof(Tile) * groups[q].t.size());
    nt += groups[q].t.size();
  }
  int32_t* hwhich = reinterpret_cast<int32_t*>(sl.host + st.which);
  if (!which.empty()) memcpy(hwhich, which.data(), sizeof(int32_t) * which.size());
  // a failure from here on hands the admitted requests back: their scratch
  // returns to the pool, their drones become idle, and they rejoin the queue
  // in arrival order (request ids grow with arrival)
  auto undo = [&](cudaError_t e, const char* what) {
    for (Request& r : batch) {
      s->pool.release(r.off, r.bytes);
      s->drones[r.drone].busy = false;
      r.t_launch = 0.0;
      s->queue.push_back(r);
    }
    std::sort(s->queue.begin(), s->queue.end(), [](const Request& a, const Request& b) { return a.id < b.id; });
    return sfail(MPPI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  };
#define SCU_UNDO(call)                  \
  do {                                  \
    cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) return undo(e_, #call); \
  } while (0)
  if (s->fail_next_launch) {
    s->fail_next_launch = false;
    return undo(cudaErrorLaunchFailure, "injected failure (mppi_server_fail_next_launch)");
  }
  cudaStream_t stm = sl.stream;
  SCU_UNDO(cudaMemcpyAsync(sl.dev, sl.host, st.total, cudaMemcpyHostToDevice, stm));
  const SolveDesc* ddesc = reinterpret_cast<const SolveDesc*>(sl.dev + st.descs);
  const Tile* dtiles = reinterpret_cast<const Tile*>(sl.dev + st.tiles);
  LaunchIO io;
  memset(&io, 0, sizeof io);
  io.x0 = reinterpret_cast<const float*>(sl.dev + st.x0);
  io.t0 = reinterpret_cast<const double*>(sl.dev + st.t0);
  io.u0 = sl.d_u0;
  io.status = sl.d_status;
  for (size_t q = 0; q < groups.size(); ++q)
    if (groups[q].gen == MPPI_NOISEGEN_KERNEL)
      SCU_UNDO(launch_noise(ddesc, dtiles + goff[q], (int)groups[q].t.size(), groups[q].block, groups[q].bf16, stm,
                            groups[q].nom, kMaxN));
  for (size_t q = 0; q < groups.size(); ++q)
    SCU_UNDO(launch_rollout(groups[q].obj, groups[q].bf16, ddesc, dtiles + goff[q], (int)groups[q].t.size(),
                            groups[q].block, groups[q].smem, io, stm, groups[q].gen, groups[q].rot));
  SCU_UNDO(launch_nominal(ddesc, reinterpret_cast<const int32_t*>(sl.dev + st.which), (int)which.size(), stm));
  SCU_UNDO(cudaEventRecord(sl.done, stm));
#undef SCU_UNDO
  sl.reqs.swap(batch);
  sl.busy = true;
  s->next_slot = (si + 1) % (int)s->slots.size();
  s->batches += 1;
  if (launched) *launched = (int32_t)sl.reqs.size();
  return MPPI_OK;
}

int mppi_server_fail_next_launch(mppi_server s) {
  if (!s) return sfail(MPPI_ERR_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->fail_next_launch = true;
  return MPPI_OK;
}

int mppi_server_poll(mppi_server s, mppi_result_t* out, int32_t cap, int32_t* n_out) {
  if (!s || (cap > 0 && !out)) return sfail(MPPI_ERR_ARG, "bad arguments");
  if (n_out) *n_out = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& sl : s->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return sfail(MPPI_ERR_CUDA, "batch failed: %s", cudaGetErrorString(q));
    const double t = now_s();
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      const Request& r = sl.reqs[i];
      mppi_result_t res;
      res.request = r.id;
      res.drone = r.drone;
      res.status = ((volatile int32_t*)sl.status)[i];
      res.K = r.K;
      res.N = r.N;
      for (int j = 0; j < kNU; ++j) res.u0[j] = ((volatile float*)sl.u0)[(size_t)kNU * i + j];
      res.t_submit = r.t_submit;
      res.t_launch = r.t_launch;
      res.t_done = t;
      s->done.push_back(res);
      s->pool.release(r.off, r.bytes);
      s->drones[r.drone].busy = false;
    }
    s->finished += (double)sl.reqs.size();
    sl.reqs.clear();
    sl.busy = false;
  }
  const int n = std::min<int>(cap, (int)s->done.size());
  if (n > 0) {
    std::copy(s->done.begin(), s->done.begin() + n, out);
    s->done.erase(s->done.begin(), s->done.begin() + n);
  }
  if (n_out) *n_out = n;
  return MPPI_OK;
}

int mppi_server_stats(mppi_server s, double out[8]) {
  if (!s || !out) return sfail(MPPI_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  double inflight = 0;
  for (auto& sl : s->slots) inflight += (double)sl.reqs.size();
  out[0] = (double)s->queue.size();
  out[1] = inflight;
  out[2] = (double)s->pool.used();
  out[3] = (double)s->pool.peak();
  out[4] = s->batches;
  out[5] = s->finished;
  out[6] = (double)s->drones.size();
  out[7] = (double)s->pool.size();
  return MPPI_OK;
}

int mppi_server_export_drone(mppi_server s, int32_t drone, void* buf, size_t* size) {
  if (!s || !size) return sfail(MPPI_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (drone < 0 || drone >= (int)s->drones.size()) return sfail(MPPI_ERR_ARG, "unknown drone");
  const Drone& d = s->drones[drone];
  const size_t need = 16 + sizeof(DevState) + sizeof(float) * d.N_cap * kNU + sizeof(int32_t) * d.N_cap;
  if (!buf) {
    *size = need;
    return MPPI_OK;
  }
  if (*size < need) return sfail(MPPI_ERR_ARG, "buffer too small");
  for (auto& sl : s->slots)
    if (sl.busy) SCU(cudaEventSynchronize(sl.done));
  char* c = static_cast<char*>(buf);
  const uint32_t hdr[4] = {0x4D505049u, 1u, (uint32_t)d.N_cap, (uint32_t)d.nu};
  memcpy(c, hdr, 16);
  c += 16;
  SCU(cudaMemcpy(c, d.hd.st, sizeof(DevState), cudaMemcpyDeviceToHost));
  c += sizeof(DevState);
  SCU(cudaMemcpy(c, d.hd.U, sizeof(float) * d.N_cap * kNU, cudaMemcpyDeviceToHost));
  c += sizeof(float) * d.N_cap * kNU;
  SCU(cudaMemcpy(c, d.hd.prevcnt, sizeof(int32_t) * d.N_cap, cudaMemcpyDeviceToHost));
  *size = need;
  return MPPI_OK;
}

int mppi_server_destroy(mppi_server s) {
  if (!s) return MPPI_OK;
  destroy_server(s);
  return MPPI_OK;
}

}  // extern "C"
