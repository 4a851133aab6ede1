// mppi_noalloc.cu -- a solve entry point that allocates nothing.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree once they are
// running.  A flight-control loop certified to do all allocation at start-up
// is one; so is a process whose GPU memory belongs to another allocator (a
// framework's caching pool), and any loop that cannot afford the implicit
// device-wide synchronisation a cudaMalloc may cause.  mppi_create allocates
// a slab per handle, so those callers cannot use the handle API on their hot
// path.  mppi_solve_noalloc runs the same noise and rollout kernels, but keeps
// every per-solve scratch buffer (descriptor, controller state, tile table,
// noise, costs, tile partials, merge tickets) in one file-scope device array
// of fixed size that is loaded with the library.
#include <cstdio>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mppi_device.cuh"
#include "mppi_launch.h"

using namespace mppi;

namespace {

// Scratch shared by every mppi_solve_noalloc call on a device.  In host code
// this name is only a stand-in for the device symbol: its address comes from
// cudaGetSymbolAddress (see scratch_on_device).
constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int fail(int code, const char* what) {
  char msg[320];
  snprintf(msg, sizeof msg, "mppi_solve_noalloc: %s", what);
  set_last_error(msg);
  return code;
}

// One-time set-up per device (that device must be current): the device
// address of the scratch array and the kernels' shared-memory limits.
int scratch_on_device(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return fail(MPPI_ERR_ARG, "device index out of range");
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
      return fail(MPPI_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    if (configure_kernels() != cudaSuccess) return fail(MPPI_ERR_CUDA, "kernel configuration failed");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MPPI_OK;
}

struct Layout {
  size_t desc, st, tiles, U, prev, gframes, Z, Z5, J, info, pm, pS, pP, ticket, passcnt, xref, total;
};

Layout layout_for(int K, int N, int block, int five, int bf16, bool stored) {
  const int T = (K + block - 1) / block;
  int sq = 1;
  while (sq * sq < T) ++sq;
  const int Gn = 2 * sq + 16;
  Layout L;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o = al256(o + b);
    return r;
  };
  L.desc = take(sizeof(SolveDesc));
  L.st = take(sizeof(DevState));
  L.tiles = take(sizeof(Tile) * T);
  L.U = take(sizeof(float) * (N * kNU + 8));
  L.prev = take(sizeof(int32_t) * (N + 8));
  L.gframes = take(sizeof(GateF) * MPPI_MAX_GATES);
  L.Z = take(stored ? (size_t)N * K * (bf16 ? 8 : 16) : 16);
  L.Z5 = take(five && stored ? (size_t)N * K * (bf16 ? 2 : 4) : 16);
  L.J = take(sizeof(double) * K);
  L.info = take(sizeof(int32_t) * K);
  L.pm = take(sizeof(double) * (T + Gn + 1));
  L.pS = take(sizeof(double) * (T + Gn + 1));
  L.pP = take(sizeof(double) * (size_t)(T + Gn + 1) * N * kNU);
  L.ticket = take(sizeof(uint32_t) * (Gn + 2));
  L.passcnt = take(sizeof(int32_t) * (N + 1));
  L.xref = take(sizeof(float) * 13 * (N + 1));
  L.total = o;
  return L;
}

// Writes the descriptor, a fresh controller state, the tile table and the
// nominal into the scratch, and clears everything that must start at zero
// (the merge tickets and the previous-pass counts): the array still holds the
// last call's values.
__global__ void noalloc_setup_kernel(SolveDesc d, SolveDesc* d_desc, const float* __restrict__ U_in, uint32_t iter,
                                     int32_t gate, int32_t n_tickets) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  if (tid == 0) {
    *d_desc = d;
    DevState s;
    memset(&s, 0, sizeof s);
    s.gate = gate;
    s.iter = iter;
    s.c_last = d.hover;
    s.n_nom = d.N;
    s.status = MPPI_OK;
    *d.st = s;
  }
  for (int i = tid; i < d.N * kNU; i += nth) d.U[i] = U_in[i];
  for (int i = tid; i < d.N; i += nth) d.prevcnt[i] = 0;
  for (int i = tid; i < n_tickets; i += nth) d.ticket[i] = 0u;
}

__global__ void noalloc_tiles_kernel(Tile* tiles, int T, int tile) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < T) tiles[i] = Tile{0, i * tile};
}

}  // namespace

extern "C" int mppi_solve_noalloc(const mppi_model_t* model, const mppi_params_t* params, const mppi_track_t* d_track,
                                  const float* d_x0, double t0, const float* d_U, uint32_t iter, int32_t gate,
                                  void* stream, float* d_Unew, float* d_u0) {
  if (!model || !params || !d_track || !d_x0 || !d_U || !d_Unew || !d_u0) return fail(MPPI_ERR_ARG, "null argument");
  const mppi_model_t& m = *model;
  const mppi_params_t& p = *params;
  if (m.kind != MPPI_MODEL_CTBR) return fail(MPPI_ERR_ARG, "only the collective-thrust/body-rate model");
  if (p.objective < 0 || p.objective > 2) return fail(MPPI_ERR_ARG, "unknown objective");
  const int block = p.block ? p.block : 128;
  if (block < 32 || block > kMaxBlock || block % 32) return fail(MPPI_ERR_ARG, "block must be a multiple of 32 in [32, 512]");
  if (p.K < 1 || p.N < 1 || p.N > MPPI_MAX_N) return fail(MPPI_ERR_ARG, "K or N out of range");
  if (!(p.dt > 0) || !(p.lambda > 0)) return fail(MPPI_ERR_ARG, "dt and lambda must be positive");
  if (p.noise_gen == MPPI_NOISEGEN_AHEAD) return fail(MPPI_ERR_ARG, "noise drawn ahead needs a handle (it outlives the call)");
  if (p.noise_gen < MPPI_NOISEGEN_KERNEL || p.noise_gen > MPPI_NOISEGEN_SMEM)
    return fail(MPPI_ERR_ARG, "unknown noise generation mode");
  if (p.noise_gen == MPPI_NOISEGEN_REGEN && p.noise_dtype != MPPI_NOISE_F32)
    return fail(MPPI_ERR_ARG, "regenerated noise is never stored: it has no bfloat16 form");
  if (p.noise_dtype != MPPI_NOISE_F32 && p.noise_dtype != MPPI_NOISE_BF16) return fail(MPPI_ERR_ARG, "noise dtype");
  if (p.samples_per_thread < 0 || p.samples_per_thread > MPPI_MAX_SPT)
    return fail(MPPI_ERR_ARG, "samples_per_thread out of range");
  if (d_track->n_gates < 0 || d_track->n_gates > MPPI_MAX_GATES) return fail(MPPI_ERR_ARG, "n_gates out of range");
  if (p.noise_gen == MPPI_NOISEGEN_SMEM) {
    const int tile = block * (p.samples_per_thread ? p.samples_per_thread : 1);
    const int rows = p.objective == MPPI_OBJ_TRACK ? ref_rows_for(p.N, p.dt, d_track->dt_ref, d_track->T) : 0;
    if (rollout_smem_bytes(p.N, p.objective, d_track->S, tile, std::max(32, (p.K + tile - 1) / tile),
                           MPPI_NOISEGEN_SMEM, rows) > kRolloutSmemMax)
      return fail(MPPI_ERR_ARG, "noise kept in shared memory does not fit a block's shared memory");
  }
  if (gate < 0) return fail(MPPI_ERR_ARG, "gate index is negative");
  if (p.objective == MPPI_OBJ_GATE && (d_track->n_gates < 1 || !d_track->gates))
    return fail(MPPI_ERR_ARG, "gate objective needs gates");
  if (p.objective == MPPI_OBJ_CONTOUR && (d_track->S < 2 || !d_track->path || !(d_track->L > 0)))
    return fail(MPPI_ERR_ARG, "contouring needs a path table");
  if (p.objective == MPPI_OBJ_TRACK && (d_track->T < 2 || !d_track->ref || !(d_track->dt_ref > 0)))
    return fail(MPPI_ERR_ARG, "tracking needs a reference table");
  const int five = p.objective == MPPI_OBJ_CONTOUR;
  const int bf16 = p.noise_dtype == MPPI_NOISE_BF16;
  // regenerated noise and noise kept in shared memory need no buffer
  const bool stored = p.noise_gen != MPPI_NOISEGEN_REGEN && p.noise_gen != MPPI_NOISEGEN_SMEM;
  const Layout L = layout_for(p.K, p.N, block, five, bf16, stored);
  if (L.total > kScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf, "K=%d, N=%d need %zu bytes of scratch, more than the %zu-byte static maximum", p.K,
             p.N, L.total, kScratchBytes);
    return fail(MPPI_ERR_ARG, buf);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(MPPI_ERR_CUDA, "cudaGetDevice failed");
  void* base = nullptr;
  int rc = scratch_on_device(dev, &base);
  if (rc) return rc;
  char* b = static_cast<char*>(base);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // descriptor (the model and weight fields that mppi_create derives, from
  // the same routine), pointing into the scratch
  SolveDesc d;
  memset(&d, 0, sizeof d);
  fill_model_params(m, p, five ? 5 : 4, d);
  d.gates = d_track->gates;
  d.gframes = reinterpret_cast<const GateF*>(b + L.gframes);
  d.n_gates = d_track->n_gates;
  d.closed = d_track->closed ? 1 : 0;
  d.path = d_track->path;
  d.S = d_track->S;
  d.L = d_track->L;
  d.ds = d_track->S > 0 ? (float)((double)d_track->L / d_track->S) : 1.f;
  d.inv_ds = d_track->S > 0 ? (float)((double)d_track->S / d_track->L) : 1.f;
  d.ref = d_track->ref;
  d.T = d_track->T;
  d.dt_ref = d_track->dt_ref;
  // the caller's reference table: staged by bulk copies only from a 16-byte
  // aligned table, and never past its end (no padding is known)
  d.ref_rows = p.objective == MPPI_OBJ_TRACK && d_track->ref && reinterpret_cast<uintptr_t>(d_track->ref) % 16 == 0
                   ? ref_rows_for(p.N, p.dt, d_track->dt_ref, d_track->T)
                   : 0;
  d.ref_pad = 0;
  d.st = reinterpret_cast<DevState*>(b + L.st);
  d.U = reinterpret_cast<float*>(b + L.U);
  d.prevcnt = reinterpret_cast<int32_t*>(b + L.prev);
  d.N_cap = p.N;
  d.Z4 = (stored && !bf16) ? reinterpret_cast<float4*>(b + L.Z) : nullptr;
  d.Zb = (stored && bf16) ? reinterpret_cast<uint2*>(b + L.Z) : nullptr;
  d.Z5 = (stored && five && !bf16) ? reinterpret_cast<float*>(b + L.Z5) : nullptr;
  d.Z5b = (stored && five && bf16) ? reinterpret_cast<__nv_bfloat16*>(b + L.Z5) : nullptr;
  d.J = reinterpret_cast<double*>(b + L.J);
  d.info = reinterpret_cast<int32_t*>(b + L.info);
  d.part_m = reinterpret_cast<double*>(b + L.pm);
  d.part_S = reinterpret_cast<double*>(b + L.pS);
  d.part_P = reinterpret_cast<double*>(b + L.pP);
  d.ticket = reinterpret_cast<uint32_t*>(b + L.ticket);
  d.unew = d_Unew;
  d.passcnt = reinterpret_cast<int32_t*>(b + L.passcnt);
  d.xref = reinterpret_cast<float*>(b + L.xref);
  d.block = block;
  d.n_tiles = (p.K + tile_samples(d) - 1) / tile_samples(d);  // at most the layout's tiles
  d.ext_noise = 0;
  int sq = 1;
  while (sq * sq < d.n_tiles) ++sq;
  const int n_tickets = 2 * sq + 18;

  SolveDesc* d_desc = reinterpret_cast<SolveDesc*>(b + L.desc);
  Tile* d_tiles = reinterpret_cast<Tile*>(b + L.tiles);
  (void)cudaGetLastError();
  noalloc_setup_kernel<<<4, 256, 0, s>>>(d, d_desc, d_U, iter, gate, n_tickets);
  noalloc_tiles_kernel<<<(d.n_tiles + 255) / 256, 256, 0, s>>>(d_tiles, d.n_tiles, tile_samples(d));
  add_launches(2);
  if (cudaGetLastError() != cudaSuccess) return fail(MPPI_ERR_CUDA, "set-up kernel launch failed");
  if (p.objective == MPPI_OBJ_GATE &&
      launch_gate_frames(d_track->gates, d_track->n_gates, const_cast<GateF*>(d.gframes), s) != cudaSuccess)
    return fail(MPPI_ERR_CUDA, "gate frame launch failed");
  if (d.noise_gen == MPPI_NOISEGEN_KERNEL &&
      launch_noise(d_desc, d_tiles, d.n_tiles, block, bf16, s, d.nominal_sample, d.N) != cudaSuccess)
    return fail(MPPI_ERR_CUDA, "noise kernel launch failed");
  LaunchIO io;
  memset(&io, 0, sizeof io);
  io.x0 = d_x0;
  io.t0 = nullptr;
  io.t0v = t0;
  io.u0 = d_u0;
  io.status = nullptr;
  const uint32_t smem =
      rollout_smem_bytes(p.N, p.objective, d.S, tile_samples(d), d.n_tiles > 32 ? d.n_tiles : 32, p.noise_gen,
                         d.ref_rows);
  if (launch_rollout(p.objective, bf16, d_desc, d_tiles, d.n_tiles, block, smem, io, s, d.noise_gen, d.rotor) !=
      cudaSuccess)
    return fail(MPPI_ERR_CUDA, "rollout kernel launch failed");
  return MPPI_OK;
}
