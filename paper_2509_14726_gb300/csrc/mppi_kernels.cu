// mppi_kernels.cu -- the sm_103a kernels of one MPPI solve (arXiv 2509.14726)
// other than the rollout (mppi_rollout.cuh), and the launch entry points.
//
//   noise_kernel     Eq. 3: Philox4x32-10 -> Box-Muller standard normals,
//                    stored [N][K] so that a warp writes 512 contiguous bytes.
//   nominal_kernel   rollout of U*_new from x0 with the gate logic: the gate
//                    pass counts that the temporal-consistency rule of the next
//                    solve reads (Sec. IV-A).
//   test kernels     Philox words, normals and plain rollouts of given
//                    sequences, for the parity tests.
#include <algorithm>
#include <atomic>

#include "mppi_rollout.cuh"

namespace mppi {

static std::atomic<unsigned long long> g_launches{0};  // host threads may launch concurrently
unsigned long long launches_so_far() { return g_launches.load(); }
void add_launches(int n) { g_launches += (unsigned long long)n; }

uint32_t rollout_smem_bytes(int N, int objective, int S, int tile, int merge_cap, int gen, int ref_rows) {
  return smem_layout(N, objective, S, tile, merge_cap, path_fits_smem(S), gen, ref_rows).total;
}

// the frame of every gate (centre, plane normal from the yaw, half sizes)
__global__ void gate_frames_kernel(const float* __restrict__ raw, int n, GateF* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* g = raw + 6 * i;
  float s, c;
  sincosf(g[3], &s, &c);
  out[i] = GateF{g[0], g[1], g[2], c, s, g[4], g[5], 0.f};
}

cudaError_t launch_gate_frames(const float* raw, int n, GateF* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  gate_frames_kernel<<<(n + 63) / 64, 64, 0, s>>>(raw, n, out);
  ++g_launches;
  return cudaGetLastError();
}

int rollout_max_block() { return MPPI_ROLLOUT_MIN_BLOCKS > 0 ? 128 : kMaxBlock; }

// ---------------------------------------------------------------------------
// K1: noise
// ---------------------------------------------------------------------------
// NOM: the launch holds solves whose sample 0 is the unperturbed nominal
// (a separate instance, so that the common launch carries no test for it).
// Block (x, y) draws tile x's normals for the y-th of gridDim.y equal spans
// of the horizon: a launch of few tiles (one small solve) is split along k so
// that it still fills the GPU; a batch of many tiles runs one span.
template <int BF16, int NOM>
__global__ void __launch_bounds__(kMaxBlock) noise_kernel(const SolveDesc* __restrict__ descs,
                                                          const Tile* __restrict__ tiles) {
  const Tile tile = tiles[blockIdx.x];
  const SolveDesc& d = descs[tile.solve];
  const int K = d.K, N = d.N;
  if (d.ext_noise || threadIdx.x >= d.block) return;
  const int span = (N + (int)gridDim.y - 1) / (int)gridDim.y;
  const int k_begin = (int)blockIdx.y * span, k_end = min(N, k_begin + span);
  if (k_begin >= k_end) return;
  const uint32_t iter = d.st->iter;
  const bool five = d.nu == 5;
  // the thread's samples: m0 + tid + r block, r < samples per thread
  for (int r = 0; r < d.spt; ++r) {
    const int m = tile.m0 + threadIdx.x + r * d.block;
    if (m >= K) return;
    if (NOM && m == 0 && d.nominal_sample) {
      // the nominal candidate (Eq. 3 with du = 0) is stored as zero normals
      for (int k = k_begin; k < k_end; ++k) {
        const size_t idx = (size_t)k * K;
        if (BF16) {
          d.Zb[idx] = make_uint2(0u, 0u);
          if (five) d.Z5b[idx] = __float2bfloat16_rn(0.f);
        } else {
          d.Z4[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (five) d.Z5[idx] = 0.f;
        }
      }
      continue;
    }
#pragma unroll kNoiseUnroll
    for (int k = k_begin; k < k_end; ++k) {
      const float4 z = normals4(d.seed, d.drone_id, (uint32_t)m, (uint32_t)k, iter, 0u);
      const size_t idx = (size_t)k * K + m;
      if (BF16) {
        __nv_bfloat162 a = __floats2bfloat162_rn(z.x, z.y), b = __floats2bfloat162_rn(z.z, z.w);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&a);
        w.y = *reinterpret_cast<uint32_t*>(&b);
        d.Zb[idx] = w;
      } else {
        d.Z4[idx] = z;
      }
      if (five && (k == k_begin || (k & 3) == 0)) {
        // contouring's 5th normals of steps 4j .. 4j+3 (those in this span):
        // the four normals of one block-1 draw (the values normal5 returns),
        // stored at once so that nothing stays live across the steps
        const int k4 = k & ~3;
        const float4 z5 = normals4(d.seed, d.drone_id, (uint32_t)m, (uint32_t)k4, iter, 1u);
        const float v5[4] = {z5.x, z5.y, z5.z, z5.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = k4 + t;
          if (j < k || j >= k_end) continue;
          const size_t jdx = (size_t)j * K + m;
          if (BF16)
            d.Z5b[jdx] = __float2bfloat16_rn(v5[t]);
          else
            d.Z5[jdx] = v5[t];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K4: nominal rollout (gate pass counts for the temporal rule of the next solve)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) nominal_kernel(const SolveDesc* __restrict__ descs,
                                                      const int32_t* __restrict__ which, int n) {
  __shared__ int sPrev[4][kMaxN];
  __shared__ GateF sG[4][kMaxGates];
  __shared__ StepConsts sSC[4];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 4 + w;
  if (i >= n) return;
  const SolveDesc& d = descs[which[i]];
  DevState* st = d.st;
  const int N = d.N;
  const int adv = st->adv;
  for (int k = lane; k < N; k += 32) sPrev[w][k] = max(0, d.prevcnt[k] - adv);
  if (lane < 2) sSC[w].c[lane] = d.stepc.c[lane];
  for (int g = lane; g < d.n_gates; g += 32) sG[w][g] = d.gframes[g];
  __syncwarp();
  int pc_last = 0;
  if (lane == 0) {
    ModelRegs M;
    M.inv_mass = d.inv_mass; M.gravity = d.gravity; M.k_omega = d.k_omega;
    M.g0 = d.gyro[0]; M.g1 = d.gyro[1]; M.g2 = d.gyro[2];
    M.d0 = d.drag[0]; M.d1 = d.drag[1]; M.d2 = d.drag[2]; M.has_drag = d.has_drag;
    const float* x0 = st->prev_x0;
    Quad s;
    quad_init(s, x0);
    const float qe0 = quat_norm_excess(x0[6], x0[7], x0[8], x0[9]);
    int gi = st->gate, passed = 0;
    GateF g = load_gate(sG[w], gate_slot(gi, d.n_gates, d.closed));
    float sa = plane_dist(g, s.px, s.py);
    d.passcnt[0] = 0;
    RotorRegs RR = rotor_regs(d);
    float Tr[4] = {st->rotor_prev[0], st->rotor_prev[1], st->rotor_prev[2], st->rotor_prev[3]};
    float Trc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < N; ++k) {
      const float* u = d.unew + kNU * k;
      const float ax = pxt(s), ay = pyt(s), az = pzt(s);
      float dpx, dpy, dpz, dT2;
      if (d.rotor) {
        if (M.has_drag)
          rk4_step_rotor<true>(M, RR, &sSC[w], s, k ? 0.f : qe0, Tr, Trc, u[0], u[1], u[2], u[3], d.dt, dpx, dpy, dpz, dT2);
        else
          rk4_step_rotor<false>(M, RR, &sSC[w], s, k ? 0.f : qe0, Tr, Trc, u[0], u[1], u[2], u[3], d.dt, dpx, dpy, dpz, dT2);
      } else if (M.has_drag) {
        rk4_step<true>(M, &sSC[w], s, k ? 0.f : qe0, u[0], u[1], u[2], u[3], d.dt, dpx, dpy, dpz);
      } else {
        rk4_step<false>(M, &sSC[w], s, k ? 0.f : qe0, u[0], u[1], u[2], u[3], d.dt, dpx, dpy, dpz);
      }
      const float bx = pxt(s), by = pyt(s), bz = pzt(s);
      const float sb = plane_dist(g, bx, by);
      if (sa < 0.f && sb >= 0.f) {
        const bool open_track_done = (d.closed == 0) && gi >= d.n_gates;
        const bool ok_time = d.temporal_rule == MPPI_RULE_OFF || sPrev[w][k] <= passed;
        if (!open_track_done && ok_time && through_opening(g, sa, sb, ax, ay, az, bx - ax, by - ay, bz - az)) {
          ++passed;
          ++gi;
          g = load_gate(sG[w], gate_slot(gi, d.n_gates, d.closed));
          sa = plane_dist(g, bx, by);
        } else {
          sa = sb;
        }
      } else {
        sa = sb;
      }
      d.passcnt[k + 1] = passed;
    }
    pc_last = passed;
  }
  __syncwarp();
  pc_last = __shfl_sync(0xffffffffu, pc_last, 0);
  // counts as seen from the next solve (time aligned: one step later)
  const int shift = d.temporal_rule == MPPI_RULE_SAME_INDEX ? 0 : 1;
  for (int k = lane; k < d.N_cap; k += 32) {
    const int src = k + shift;
    d.prevcnt[k] = src <= N ? d.passcnt[src] : pc_last;
  }
  if (lane == 0) st->n_prev = N;
}

// ---------------------------------------------------------------------------
// test entry kernels
// ---------------------------------------------------------------------------
__global__ void philox_kernel(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                              uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 x = philox4x32_10(make_uint4(c0 + (uint32_t)i, c1, c2, c3), k0, k1);
  reinterpret_cast<uint4*>(out)[i] = x;
}

__global__ void normals_kernel(uint32_t seed, uint32_t drone, uint32_t k, uint32_t it, uint32_t blk, int n,
                               float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  reinterpret_cast<float4*>(out)[i] = normals4(seed, drone, (uint32_t)i, k, it, blk);
}

// rotor (rotor model): T0 [B][4] start thrusts, Tout [B][N+1][4] thrusts
__global__ void rollout_states_kernel(ModelRegs M, RotorRegs R, StepConsts SC, int rotor, float dt, int N, int B,
                                      const float* __restrict__ x0, const float* __restrict__ U,
                                      float* __restrict__ X, const float* __restrict__ T0,
                                      float* __restrict__ Tout) {
  __shared__ StepConsts sSC;
  if (threadIdx.x < 2) sSC.c[threadIdx.x] = SC.c[threadIdx.x];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float T[4] = {0.f, 0.f, 0.f, 0.f}, Tc[4] = {0.f, 0.f, 0.f, 0.f};
  if (rotor) {
    for (int r = 0; r < 4; ++r) {
      T[r] = T0[(size_t)b * 4 + r];
      Tout[(size_t)b * (N + 1) * 4 + r] = T[r];
    }
  }
  Quad s;
  quad_init(s, x0);
  const float qe0 = quat_norm_excess(x0[6], x0[7], x0[8], x0[9]);
  float* o = X + (size_t)b * (N + 1) * kNX;
  for (int c = 0; c < kNX; ++c) o[c] = x0[c];
  for (int k = 0; k < N; ++k) {
    const float* u = U + ((size_t)b * N + k) * 4;
    float dpx, dpy, dpz, dT2;
    if (rotor) {
      if (M.has_drag)
        rk4_step_rotor<true>(M, R, &sSC, s, k ? 0.f : qe0, T, Tc, u[0], u[1], u[2], u[3], dt, dpx, dpy, dpz, dT2);
      else
        rk4_step_rotor<false>(M, R, &sSC, s, k ? 0.f : qe0, T, Tc, u[0], u[1], u[2], u[3], dt, dpx, dpy, dpz, dT2);
      for (int c = 0; c < 4; ++c) Tout[((size_t)b * (N + 1) + k + 1) * 4 + c] = T[c] - Tc[c];
    } else if (M.has_drag) {
      rk4_step<true>(M, &sSC, s, k ? 0.f : qe0, u[0], u[1], u[2], u[3], dt, dpx, dpy, dpz);
    } else {
      rk4_step<false>(M, &sSC, s, k ? 0.f : qe0, u[0], u[1], u[2], u[3], dt, dpx, dpy, dpz);
    }
    float* r = o + (size_t)(k + 1) * kNX;
    r[0] = pxt(s); r[1] = pyt(s); r[2] = pzt(s);
    r[3] = s.vx - s.cvx; r[4] = s.vy - s.cvy; r[5] = s.vz - s.cvz;
    r[6] = s.qw - s.cqw; r[7] = s.qx - s.cqx; r[8] = s.qy - s.cqy; r[9] = s.qz - s.cqz;
    r[10] = s.wx - s.cwx; r[11] = s.wy - s.cwy; r[12] = s.wz - s.cwz;
  }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------

// spans of the horizon per tile: enough blocks for two per SM, at most one
// span per step of the longest horizon
static int noise_spans(int n_tiles, int N_max) {
  static const int n_sm = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 0;
    (void)cudaGetLastError();
    return v > 0 ? v : 1;
  }();
  const int want = (2 * n_sm + n_tiles - 1) / n_tiles;
  return std::max(1, std::min(want, std::max(1, N_max)));
}

cudaError_t launch_noise(const SolveDesc* descs, const Tile* tiles, int n_tiles, int block, int bf16,
                         cudaStream_t s, int nominal, int N_max) {
  if (n_tiles <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  const dim3 grid((unsigned)n_tiles, (unsigned)noise_spans(n_tiles, N_max));
  if (bf16)
    nominal ? noise_kernel<1, 1><<<grid, block, 0, s>>>(descs, tiles)
            : noise_kernel<1, 0><<<grid, block, 0, s>>>(descs, tiles);
  else
    nominal ? noise_kernel<0, 1><<<grid, block, 0, s>>>(descs, tiles)
            : noise_kernel<0, 0><<<grid, block, 0, s>>>(descs, tiles);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t configure_kernels() {
  cudaError_t e = configure_rollout_gate();
  if (e == cudaSuccess) e = configure_rollout_contour();
  if (e == cudaSuccess) e = configure_rollout_track();
  return e;
}

cudaError_t launch_rollout(int objective, int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles,
                           int block, uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor) {
  if (n_tiles <= 0) return cudaSuccess;
  switch (objective) {
    case MPPI_OBJ_GATE: return launch_rollout_gate(bf16, descs, tiles, n_tiles, block, smem, io, s, gen, rotor);
    case MPPI_OBJ_CONTOUR: return launch_rollout_contour(bf16, descs, tiles, n_tiles, block, smem, io, s, gen, rotor);
    case MPPI_OBJ_TRACK: return launch_rollout_track(bf16, descs, tiles, n_tiles, block, smem, io, s, gen, rotor);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_nominal(const SolveDesc* descs, const int32_t* which, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  nominal_kernel<<<(n + 3) / 4, 128, 0, s>>>(descs, which, n);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                          uint32_t* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  philox_kernel<<<(n + 127) / 128, 128, 0, s>>>(k0, k1, c0, c1, c2, c3, n, out);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_normals(uint32_t seed, uint32_t drone, uint32_t k, uint32_t it, uint32_t blk, int n, float* out,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  normals_kernel<<<(n + 127) / 128, 128, 0, s>>>(seed, drone, k, it, blk, n, out);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_rollout_states(const SolveDesc& md, float dt, int N, int B, const float* x0, const float* U,
                                  float* X, cudaStream_t s, const float* T0, float* Tout) {
  if (B <= 0) return cudaSuccess;
  ModelRegs M;
  M.inv_mass = md.inv_mass; M.gravity = md.gravity; M.k_omega = md.k_omega;
  M.g0 = md.gyro[0]; M.g1 = md.gyro[1]; M.g2 = md.gyro[2];
  M.d0 = md.drag[0]; M.d1 = md.drag[1]; M.d2 = md.drag[2]; M.has_drag = md.has_drag;
  RotorRegs R = rotor_regs(md);
  (void)cudaGetLastError();
  rollout_states_kernel<<<(B + 127) / 128, 128, 0, s>>>(M, R, md.stepc, md.rotor, dt, N, B, x0, U, X, T0, Tout);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace mppi
