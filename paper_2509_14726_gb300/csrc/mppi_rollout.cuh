// mppi_rollout.cuh -- the rollout kernel of one MPPI solve and the device
// code it shares with the other kernels (arXiv 2509.14726), for sm_103a.
//
//   rollout_kernel   Eq. 2 + Eq. 6-9: a thread rolls out one sample at a time
//                    (one or more per thread), RK4 in registers, objective and
//                    feasibility penalty per step; then Eq. 4/5 in
//                    flash-softmax form: each block reduces its samples to
//                    (local min cost, sum of exp weights, weighted deviation
//                    sums per (step, input)) and the last block of a group /
//                    of the solve merges those partials, writes U*_new and
//                    u0, shifts the nominal (warm start) and advances the
//                    controller state.  No grid-wide wait: an atomic ticket
//                    picks the merging block.
// The kernel template is instantiated per objective in its own translation
// unit (mppi_rollout_{gate,contour,track}.cu), which compile in parallel.
#pragma once
#include <cfloat>
#include <cmath>

#include "mppi_device.cuh"
#include "mppi_launch.h"

namespace mppi {

// loop unrolling of the per-step loops (build options)
#ifndef MPPI_NOISE_UNROLL
#define MPPI_NOISE_UNROLL 1
#endif
#ifndef MPPI_ROLLOUT_UNROLL
#define MPPI_ROLLOUT_UNROLL 1
#endif
constexpr int kNoiseUnroll = MPPI_NOISE_UNROLL;
constexpr int kRolloutUnroll = MPPI_ROLLOUT_UNROLL;

// bounded wait on an mbarrier phase; returns false after ~timeout_ns
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// TMA bulk copy global -> shared (16-byte aligned, size multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}

__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide reductions through a small shared scratch (>= 32 doubles)
__device__ inline double block_min_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_min_d(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = INFINITY;
  for (int i = 0; i < nw; ++i) r = fmin(r, red[i]);
  return r;
}
__device__ inline double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < nw; ++i) r += red[i];  // fixed order: deterministic
  return r;
}

// Binary32 forms of the block reductions.  On this GPU a dependent FP64
// operation costs about ten times the latency of an FP32 one, and these
// reductions sit on every block's critical path, so the default accumulation
// modes keep the tile minimum in binary32 and the sums as compensated
// (hi, lo) binary32 pairs; the MPPI_ACC_F64 mode keeps FP64 throughout.
// (h, l) += (h2, l2) with TwoSum, renormalised
__device__ __forceinline__ void add2(float& h, float& l, float h2, float l2) {
  float s, e;
  two_sum(h, h2, s, e);
  const float t = e + l + l2;
  two_sum(s, t, h, l);
}
__device__ __forceinline__ void warp_sum2_f(float& h, float& l) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    add2(h, l, h2, l2);
  }
}
__device__ inline float block_min_f(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_min_f(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float r = INFINITY;
  for (int i = 0; i < nw; ++i) r = fminf(r, red[i]);
  return r;
}
// block total of (h, l) pairs in a fixed order (deterministic); red holds >= 64 floats
__device__ inline void block_sum2_f(float& h, float& l, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  warp_sum2_f(h, l);
  __syncthreads();
  if (lane == 0) {
    red[2 * wid] = h;
    red[2 * wid + 1] = l;
  }
  __syncthreads();
  h = red[0];
  l = red[1];
  for (int i = 1; i < nw; ++i) add2(h, l, red[2 * i], red[2 * i + 1]);
}
__device__ __forceinline__ double pack2(float h, float l) {
  float2 r = make_float2(h, l);
  return *reinterpret_cast<double*>(&r);
}
__device__ __forceinline__ float2 unpack2(double raw) { return *reinterpret_cast<const float2*>(&raw); }

// ---------------------------------------------------------------------------
// gate geometry (Sec. IV-A): s = n . (p - c); a pass goes from s < 0 to s >= 0
// through the opening (lateral |l . e| <= half_w, vertical |e_z| <= half_h)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float plane_dist(const GateF& g, float x, float y) {
  return g.nx * (x - g.cx) + g.ny * (y - g.cy);
}

__device__ __forceinline__ bool through_opening(const GateF& g, float sa, float sb, float ax, float ay, float az,
                                                float dx, float dy, float dz) {
  const float a = sa / (sa - sb);
  const float ex = ax + a * dx - g.cx, ey = ay + a * dy - g.cy, ez = az + a * dz - g.cz;
  const float lat = -g.ny * ex + g.nx * ey;
  return fabsf(lat) <= g.hw && fabsf(ez) <= g.hh;
}

// A gate frame read from shared memory as two 16-byte vectors into scalar
// fields.  (A whole-struct copy from a dynamically indexed element was kept
// as a stack object and read back from local memory at every use.)
__device__ __forceinline__ GateF load_gate(const GateF* table, int i) {
  const float4* p = reinterpret_cast<const float4*>(table + i);
  const float4 a = p[0], b = p[1];
  GateF g;
  g.cx = a.x; g.cy = a.y; g.cz = a.z; g.nx = a.w;
  g.ny = b.x; g.hw = b.y; g.hh = b.z; g.pad = b.w;
  return g;
}

// table row of absolute gate index idx: modulo n on a closed track; on an
// open track the last gate stays targeted (and a negative index, which the
// host API refuses, reads row 0 rather than outside the table)
__device__ __forceinline__ int gate_slot(int idx, int n, int closed) {
  if (closed) {
    int r = idx % n;
    return r < 0 ? r + n : r;
  }
  return idx < 0 ? 0 : (idx < n ? idx : n - 1);
}

// ---------------------------------------------------------------------------
// shared-memory layout of the rollout kernel
// ---------------------------------------------------------------------------
struct SmemLayout {
  uint32_t off_U, off_prev, off_gates, off_path, off_xref, off_ref, off_e, off_j, off_merge, off_fin, off_z, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// tile: samples per tile (threads per block x samples per thread); gen: where
// the normals are drawn (MPPI_NOISEGEN_SMEM keeps the tile's normals here)
// ref_rows: reference rows a tracking block stages (0: none)
__host__ __device__ inline SmemLayout smem_layout(int N, int objective, int S, int tile, int merge_cap,
                                                  int path_in_smem, int gen, int ref_rows) {
  SmemLayout L;
  uint32_t o = 0;
  L.off_U = o;
  o += align16((uint32_t)N * kNU * 4u);
  L.off_prev = o;
  o += align16((uint32_t)N * 4u);
  L.off_gates = o;
  o += align16((uint32_t)kMaxGates * sizeof(GateF));
  L.off_path = o;
  if (objective == MPPI_OBJ_CONTOUR && path_in_smem) o += align16((uint32_t)S * 6u * 4u);
  L.off_xref = o;
  if (objective == MPPI_OBJ_TRACK) o += align16((uint32_t)(N + 1) * kNX * 4u) + align16((uint32_t)(N + 1) * 16u);
  L.off_ref = o;  // staged reference rows: two segments, each from a 16-byte boundary
  if (objective == MPPI_OBJ_TRACK && ref_rows > 0) o += align16((uint32_t)ref_rows * 52u + 16u) + 16u;
  L.off_e = o;
  o += align16((uint32_t)tile * 4u);
  L.off_j = o;  // the tile's costs as compensated pairs: [tile] hi, then [tile] lo
  o += align16((uint32_t)tile * 8u);
  L.off_merge = o;
  o += align16((uint32_t)merge_cap * 8u);
  L.off_z = o;  // [N][tile] float4 normals, then [N][tile] 5th normals (contouring)
  if (gen == MPPI_NOISEGEN_SMEM)
    o += align16((uint32_t)N * tile * 16u) + (objective == MPPI_OBJ_CONTOUR ? align16((uint32_t)N * tile * 4u) : 0u);
  L.off_fin = o;  // the final merge's sums of Eq. 5, [N][5] pairs (last block only)
  o += align16((uint32_t)N * kNU * 8u);
  L.total = o;
  return L;
}

__host__ __device__ inline int path_fits_smem(int S) { return S > 0 && S * 24 <= 96 * 1024; }



// NC: read through the non-coherent (read-only) path; only for noise written
// by an earlier kernel.  Noise this kernel wrote itself is read coherently.
template <int BF16, bool NC = true>
__device__ __forceinline__ void load_noise(const SolveDesc& d, size_t idx, float z[kNU], bool five) {
  if (BF16) {
    const uint2 w = NC ? __ldg(d.Zb + idx) : d.Zb[idx];
    __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
    __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    z[0] = fa.x; z[1] = fa.y; z[2] = fb.x; z[3] = fb.y;
    z[4] = five ? __bfloat162float(d.Z5b[idx]) : 0.f;
  } else {
    const float4 v = NC ? __ldg(d.Z4 + idx) : d.Z4[idx];
    z[0] = v.x; z[1] = v.y; z[2] = v.z; z[3] = v.w;
    z[4] = five ? (NC ? __ldg(d.Z5 + idx) : d.Z5[idx]) : 0.f;
  }
}

// Generates the standard normals of (sample m, step k) with the noise
// kernel's Philox / Box-Muller arithmetic and returns them.  STORE: also
// writes them (float32 or bfloat16, the values returned) for the epilogue and
// the diagnostics; without STORE the epilogue draws them again.
template <int BF16, bool STORE = true>
__device__ __forceinline__ void gen_noise(const SolveDesc& d, uint32_t iter, int m, int k, float z[kNU], bool five) {
  const size_t idx = (size_t)k * d.K + m;
  float4 v = normals4(d.seed, d.drone_id, (uint32_t)m, (uint32_t)k, iter, 0u);
  float z5 = 0.f;
  if (five) z5 = normal5(d.seed, d.drone_id, (uint32_t)m, (uint32_t)k, iter);
  if (m == 0 && d.nominal_sample) {  // Eq. 3 with du = 0
    v = make_float4(0.f, 0.f, 0.f, 0.f);
    z5 = 0.f;
  }
  if (BF16) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    if (STORE) {
      uint2 w;
      w.x = *reinterpret_cast<uint32_t*>(&a);
      w.y = *reinterpret_cast<uint32_t*>(&b);
      d.Zb[idx] = w;
    }
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    v = make_float4(fa.x, fa.y, fb.x, fb.y);
    if (five) {
      const __nv_bfloat16 h = __float2bfloat16_rn(z5);
      if (STORE) d.Z5b[idx] = h;
      z5 = __bfloat162float(h);
    }
  } else if (STORE) {
    d.Z4[idx] = v;
    if (five) d.Z5[idx] = z5;
  }
  z[0] = v.x; z[1] = v.y; z[2] = v.z; z[3] = v.w; z[4] = z5;
}

// ---------------------------------------------------------------------------
// flash-softmax merge of partials (Eq. 4 / Eq. 5 in split form):
//   m = min m_i, s_i = exp(-(m_i - m) / lambda), S = sum S_i s_i,
//   P = sum P_i s_i.  Binary32 minimum and scales with S and P as
//   compensated (hi, lo) pairs, or FP64 throughout (MPPI_ACC_F64).
// ---------------------------------------------------------------------------
struct MergeIn {
  const double* m;   // [n]
  const double* S;   // [n]
  const double* P;   // [n][NNU] (float2 hi/lo or double)
};

// PRE: partials of the thread's first output requested up front (0: none;
// the instances that would spill with them leave them out)
template <int PRE>
__device__ inline void merge_partials(const SolveDesc& d, const MergeIn in, int n, int NNU, double* out_m, double* out_S,
                               double* out_P, double* scale_s, double* red, int f64) {
  if (!f64) {
    // binary32 minimum and scales; S and P as compensated (hi, lo) pairs
    float* redf = reinterpret_cast<float*>(red);
    float* scale_f = reinterpret_cast<float*>(scale_s);
    // One round trip to L2 for the common case: the thread's own (m_i, S_i)
    // and the first PRE partials of its first output are requested before
    // the first reduction, and arrive while the minimum and the scales are
    // formed.  The sums keep the index order of the loops below.
    constexpr int kPre = PRE > 0 ? PRE : 1;
    float2 pre[kPre];
    if (PRE > 0 && (int)threadIdx.x < NNU) {
#pragma unroll
      for (int t = 0; t < kPre; ++t)
        pre[t] = t < n ? unpack2(__ldcg(in.P + (size_t)t * NNU + threadIdx.x)) : make_float2(0.f, 0.f);
    }
    const bool own = PRE > 0 && (int)threadIdx.x < n;
    const float m_own = own ? (float)__ldcg(in.m + threadIdx.x) : INFINITY;
    const float2 S_own = own ? unpack2(__ldcg(in.S + threadIdx.x)) : make_float2(0.f, 0.f);
    float mloc = m_own;
    for (int i = threadIdx.x + (PRE > 0 ? blockDim.x : 0); i < n; i += blockDim.x)
      mloc = fminf(mloc, (float)__ldcg(in.m + i));
    const float mm = block_min_f(mloc, redf);
    float sh = 0.f, sl = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float mi = own && i == (int)threadIdx.x ? m_own : (float)__ldcg(in.m + i);
      const float sc = (isinf(mm) || isinf(mi)) ? 0.f : expf(-(mi - mm) * d.inv_lambda);
      scale_f[i] = sc;
      const float2 Si = own && i == (int)threadIdx.x ? S_own : unpack2(__ldcg(in.S + i));
      const float p = Si.x * sc;
      add2(sh, sl, p, fmaf(Si.x, sc, -p) + Si.y * sc);
    }
    block_sum2_f(sh, sl, redf);  // its barriers make scale_f visible
    // further partials are requested 8 at a time (one L2 round trip per 8
    // instead of per partial) and summed in index order
    auto acc_one = [&](float& hi, float& lo, float2 v, float sc) {
      const float p = v.x * sc;
      float t, e;
      two_sum(hi, p, t, e);
      hi = t;
      lo += e + fmaf(v.x, sc, -p) + v.y * sc;
    };
    for (int o = threadIdx.x; o < NNU; o += blockDim.x) {
      float hi = 0.f, lo = 0.f;
      int i = 0;
      if (PRE > 0 && o == (int)threadIdx.x) {
#pragma unroll
        for (int t = 0; t < kPre; ++t)
          if (t < n) acc_one(hi, lo, pre[t], scale_f[t]);
        i = min(n, kPre);
      }
      for (; i + 8 <= n; i += 8) {
        float2 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = unpack2(__ldcg(in.P + (size_t)(i + t) * NNU + o));
#pragma unroll
        for (int t = 0; t < 8; ++t) acc_one(hi, lo, v[t], scale_f[i + t]);
      }
      for (; i < n; ++i) acc_one(hi, lo, unpack2(__ldcg(in.P + (size_t)i * NNU + o)), scale_f[i]);
      float t, e;
      two_sum(hi, lo, t, e);
      out_P[o] = pack2(t, e);
    }
    if (threadIdx.x == 0) {
      *out_m = (double)mm;
      *out_S = pack2(sh, sl);
    }
    return;
  }
  double mloc = INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mloc = fmin(mloc, __ldcg(in.m + i));
  const double mm = block_min_d(mloc, red);
  double sloc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double mi = __ldcg(in.m + i);
    const double s = (isinf(mm) || isinf(mi)) ? 0.0 : exp(-(mi - mm) * (double)d.inv_lambda);
    scale_s[i] = s;
    sloc += __ldcg(in.S + i) * s;
  }
  const double SS = block_sum_d(sloc, red);  // ends with __syncthreads: scale_s visible
  for (int o = threadIdx.x; o < NNU; o += blockDim.x) {
    if (f64) {
      double acc = 0.0;
      int i = 0;
      for (; i + 8 <= n; i += 8) {
        double v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = __ldcg(in.P + (size_t)(i + t) * NNU + o);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc = fma(v[t], scale_s[i + t], acc);
      }
      for (; i < n; ++i) acc = fma(__ldcg(in.P + (size_t)i * NNU + o), scale_s[i], acc);
      out_P[o] = acc;
    } else {
      float hi = 0.f, lo = 0.f;
      for (int i = 0; i < n; ++i) {
        const double raw = __ldcg(in.P + (size_t)i * NNU + o);
        const float2 v = *reinterpret_cast<const float2*>(&raw);
        const float s = (float)scale_s[i];
        // TwoProd(v.x, s) and TwoSum into (hi, lo)
        const float p = v.x * s;
        const float pe = fmaf(v.x, s, -p);
        float t, e;
        two_sum(hi, p, t, e);
        hi = t;
        lo += e + pe + v.y * s;
      }
      float t, e;
      two_sum(hi, lo, t, e);
      float2 r = make_float2(t, e);
      out_P[o] = *reinterpret_cast<double*>(&r);
    }
  }
  if (threadIdx.x == 0) {
    *out_m = mm;
    *out_S = SS;
  }
}

// ---------------------------------------------------------------------------
// K2: rollout + cost + per-block weights + merge (last block)
// ---------------------------------------------------------------------------
// Occupancy of the rollout kernel is register-bound; MPPI_ROLLOUT_MIN_BLOCKS
// (build option) caps the registers so that this many 128-thread blocks fit
// on an SM (blocks are then limited to 128 threads).  The rotor model's
// contouring instance gets one block less: at the common bound it spills,
// and with the registers of four blocks it runs 11 % faster.
#ifndef MPPI_ROLLOUT_MIN_BLOCKS
#define MPPI_ROLLOUT_MIN_BLOCKS 0
#endif
#if MPPI_ROLLOUT_MIN_BLOCKS > 0
#define MPPI_ROLLOUT_BOUNDS \
  __launch_bounds__(128, (ROT && OBJ == MPPI_OBJ_CONTOUR && MPPI_ROLLOUT_MIN_BLOCKS > 4) ? 4 : MPPI_ROLLOUT_MIN_BLOCKS)
#else
#define MPPI_ROLLOUT_BOUNDS __launch_bounds__(kMaxBlock)
#endif


// lanes that share one step in the epilogue's weighted sums (power of two <= 32)
#ifndef MPPI_EPI_BATCH
#define MPPI_EPI_BATCH 4
#endif
static_assert(MPPI_EPI_BATCH >= 1 && MPPI_EPI_BATCH <= 16, "MPPI_EPI_BATCH must be in [1, 16]");
#ifndef MPPI_EPI_LANES
#define MPPI_EPI_LANES 4
#endif
static_assert(MPPI_EPI_LANES >= 1 && MPPI_EPI_LANES <= 32 && (MPPI_EPI_LANES & (MPPI_EPI_LANES - 1)) == 0,
              "MPPI_EPI_LANES must be a power of two in [1, 32]");

// The tile's Eq. 5 sums: P[k][j] = sum_m w_m (u_mkj - U*_kj) for the block's
// samples (weights sE relative to the tile minimum), written to myP [N][5] as
// compensated (hi, lo) pairs (FP64 in MPPI_ACC_F64).  Each warp takes
// kEpiRows steps at a time with kEpiLanes lanes per step: a lane sums every
// kEpiLanes-th sample of the tile, then the lanes of a step reduce in a fixed
// order (log2(kEpiLanes) TwoSum levels).  A lane requests the weights and
// normals of kEpiBatch samples before it uses the first (a lone block
// otherwise waits one L2 latency per sample); in the compensated mode the
// batch's products form one FMA chain that enters the running sum with one
// Kahan step (the chain's rounding is a few ulps of its own few terms).
template <int ACC, int BF16, int GEN>
__device__ __forceinline__ void eq5_rows(const SolveDesc& d, const float* sU, const float* sE, uint32_t iter,
                                         int m0, int nvalid, double* myP, const float4* sZ4, const float* sZ5,
                                         int TS) {
  constexpr int kEpiLanes = MPPI_EPI_LANES, kEpiRows = 32 / kEpiLanes, kEpiBatch = GEN == 2 ? 1 : MPPI_EPI_BATCH;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const int sub = lane / kEpiLanes, sl = lane % kEpiLanes;
  const int N = d.N, K = d.K, nu = d.nu;
  const bool five = nu == 5;
  for (int k0 = wid * kEpiRows; k0 < N; k0 += nw * kEpiRows) {
    const int k = k0 + sub;
    const bool row_ok = k < N;
    const float* Uk = sU + kNU * (row_ok ? k : 0);
    float Ukj[kNU], sg[kNU], lob[kNU], hib[kNU];
#pragma unroll
    for (int j = 0; j < kNU; ++j) {
      Ukj[j] = Uk[j];
      sg[j] = d.sigma[j];
      lob[j] = d.u_min[j];
      hib[j] = d.u_max[j];
    }
    float hi[kNU], lo[kNU];
    double dacc[kNU];
#pragma unroll
    for (int j = 0; j < kNU; ++j) {
      hi[j] = 0.f;
      lo[j] = 0.f;
      if (ACC == MPPI_ACC_F64) dacc[j] = 0.0;
    }
    if (row_ok) {
      for (int i0 = sl; i0 < nvalid; i0 += kEpiBatch * kEpiLanes) {
        float wb[kEpiBatch], zb[kEpiBatch][kNU];
#pragma unroll
        for (int t = 0; t < kEpiBatch; ++t) {
          const int ic = min(i0 + t * kEpiLanes, nvalid - 1);  // in range; weight 0 past nvalid
          wb[t] = i0 + t * kEpiLanes < nvalid ? sE[ic] : 0.f;
          if (GEN == 3) {
            const float4 v = sZ4[(size_t)k * TS + ic];
            zb[t][0] = v.x; zb[t][1] = v.y; zb[t][2] = v.z; zb[t][3] = v.w;
            zb[t][4] = five ? sZ5[(size_t)k * TS + ic] : 0.f;
          } else if (GEN == 2) {
            gen_noise<BF16, false>(d, iter, m0 + ic, k, zb[t], five);
          } else {
            load_noise<BF16, GEN == 0>(d, (size_t)k * K + m0 + ic, zb[t], five);
          }
        }
        float part[kNU];
#pragma unroll
        for (int j = 0; j < kNU; ++j) part[j] = 0.f;
#pragma unroll
        for (int t = 0; t < kEpiBatch; ++t) {
          const float w = wb[t];
#pragma unroll
          for (int j = 0; j < kNU; ++j) {
            if (j >= nu) break;
            const float dv = clampf(Ukj[j] + sg[j] * zb[t][j], lob[j], hib[j]) - Ukj[j];
            if (ACC == MPPI_ACC_F64)
              dacc[j] = fma((double)w, (double)dv, dacc[j]);
            else if (ACC == MPPI_ACC_F32)
              hi[j] = fmaf(w, dv, hi[j]);
            else
              part[j] = fmaf(w, dv, part[j]);
          }
        }
        if (ACC == MPPI_ACC_KAHAN32) {
#pragma unroll
          for (int j = 0; j < kNU; ++j)
            if (j < nu) kahan_add(hi[j], lo[j], part[j]);
        }
      }
    }
    // cross-lane reduction within the step's lane group, fixed order
    const bool writer = row_ok && sl == 0;
#pragma unroll
    for (int j = 0; j < kNU; ++j) {
      if (j >= nu) break;
      if (ACC == MPPI_ACC_F64) {
        double v = dacc[j];
#pragma unroll
        for (int o = kEpiLanes / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (writer) myP[kNU * k + j] = v;
      } else if (ACC == MPPI_ACC_F32) {
        float v = hi[j];
#pragma unroll
        for (int o = kEpiLanes / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (writer) myP[kNU * k + j] = pack2(v, 0.f);
      } else {
        float h1 = hi[j], l1 = -lo[j];
#pragma unroll
        for (int o = kEpiLanes / 2; o; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, h1, o), l2 = __shfl_xor_sync(0xffffffffu, l1, o);
          add2(h1, l1, h2, l2);
        }
        if (writer) myP[kNU * k + j] = pack2(h1, l1);
      }
    }
    if (writer)
      for (int j = nu; j < kNU; ++j) myP[kNU * k + j] = ACC == MPPI_ACC_F64 ? 0.0 : pack2(0.f, 0.f);
  }
}

// ROT: rotor-thrust-rate input model (rotor thrusts in the state)
template <int OBJ, int BF16, int GEN, int ROT>
__global__ void MPPI_ROLLOUT_BOUNDS rollout_kernel(const SolveDesc* __restrict__ descs,
                                                            const Tile* __restrict__ tiles, LaunchIO io) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) SolveDesc sd;
  __shared__ __align__(8) uint64_t mbar, mbar_never;
  __shared__ double red[32];
  __shared__ float x0s[kNX];
  // (sigma, u_min, u_max, 0) per input; (w_limit, omega_max, z_floor, 0);
  // (q_near, r_near^2, 0, 0)
  __shared__ float4 sBnd[6];
  __shared__ int s_adv, s_last, s_group_last, s_bad, s_gate0, s_slot0;
  __shared__ double s_theta0, s_m, s_S;
  __shared__ float s_vth0, s_f0, s_qe0, s_rf0;
  __shared__ float2 s_rr;
  __shared__ int s_j0, s_ri0, s_win[2];
  // staged reference rows: rows before the wrap, first row's byte offset in
  // its 16-byte-aligned copy, offset of the second copy, copy sizes, source
  __shared__ int s_ref_n1, s_ref_lead, s_ref_seg2;
  __shared__ uint32_t s_ref_len[2], s_ref_src;
  __shared__ float s_best_d[32];
  __shared__ int s_best_j[32];
  __shared__ float s_best_t[32];

  const Tile tile = tiles[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  {
    const int* src = reinterpret_cast<const int*>(descs + tile.solve);
    int* dst = reinterpret_cast<int*>(&sd);
    for (int i = tid; i < (int)(sizeof(SolveDesc) / 4); i += blockDim.x) dst[i] = src[i];
  }
  if (tid < kNX) x0s[tid] = io.x0 ? io.x0[(size_t)tile.solve * kNX + tid] : io.x0v[tid];
  __syncthreads();
  const SolveDesc& d = sd;
  if (tid == 0) s_qe0 = quat_norm_excess(x0s[6], x0s[7], x0s[8], x0s[9]);
  if (tid < 4) sBnd[tid] = make_float4(d.sigma[tid], d.u_min[tid], d.u_max[tid], 0.f);
  if (tid == 4) sBnd[4] = make_float4(d.w_limit, d.omega_max, d.z_floor, 0.f);
  if (tid == 5) sBnd[5] = make_float4(d.q_near, d.r_near2, 0.f, 0.f);
  const int K = d.K, N = d.N, nu = d.nu, B = d.block;
  const int path_smem = path_fits_smem(d.S);
  // the tile: TS = B spt samples; thread tid runs m0 + tid + rep B, rep < spt
  const int spt = d.spt, TS = B * spt;
  const SmemLayout Ls = smem_layout(N, OBJ, d.S, TS, max(d.n_tiles, 32), path_smem, GEN, d.ref_rows);
  // GEN 3: the tile's normals, kept here for the update (Eq. 5)
  float4* sZ4 = reinterpret_cast<float4*>(smem + Ls.off_z);
  float* sZ5 = reinterpret_cast<float*>(smem + Ls.off_z + align16((uint32_t)N * TS * 16u));
  float* sU = reinterpret_cast<float*>(smem + Ls.off_U);
  int* sPrev = reinterpret_cast<int*>(smem + Ls.off_prev);
  GateF* sG = reinterpret_cast<GateF*>(smem + Ls.off_gates);
  float* sPath = path_smem ? reinterpret_cast<float*>(smem + Ls.off_path) : nullptr;
  float* sX = reinterpret_cast<float*>(smem + Ls.off_xref);           // [N+1][13]
  float* sXl = sX + align16((uint32_t)(N + 1) * kNX * 4u) / 4;          // [N+1][4] low parts of p
  float* sE = reinterpret_cast<float*>(smem + Ls.off_e);
  float* sJ = reinterpret_cast<float*>(smem + Ls.off_j);  // [TS] hi (NaN: not valid), [TS] lo
  double* sMerge = reinterpret_cast<double*>(smem + Ls.off_merge);
  const float* path = path_smem ? sPath : d.path;

  // ---- prologue: TMA bulk copies into shared memory of the nominal, the
  // gate frames (gate progress), the path table (contouring) and the span of
  // reference rows the tracking window reads ----
  const uint32_t bytes_U = align16((uint32_t)N * kNU * 4u);
  const uint32_t bytes_path = (OBJ == MPPI_OBJ_CONTOUR && path_smem) ? align16((uint32_t)d.S * 24u) : 0u;
  const uint32_t bytes_gates = OBJ == MPPI_OBJ_GATE ? (uint32_t)d.n_gates * (uint32_t)sizeof(GateF) : 0u;
  unsigned char* sRef = smem + Ls.off_ref;
  DevState* st = d.st;
  if (tid == 0) {
    mbar_init(&mbar, 1);
    if (d.wait_unreachable) mbar_init(&mbar_never, 1);
    s_bad = 0;
    uint32_t bytes_ref = 0;
    if (OBJ == MPPI_OBJ_TRACK) {
      // the time origin as a table position (row i0, fraction f0), once per
      // block; the step positions f0 + k dt/dt_ref are formed below in
      // binary32 with dt/dt_ref as a (hi, lo) pair
      const double t0 = io.t0 ? io.t0[tile.solve] : io.t0v;
      const double period = (double)d.T * (double)d.dt_ref;
      double tau = fmod(t0, period);
      if (tau < 0) tau += period;
      const double s0 = tau / (double)d.dt_ref;
      const double fi = floor(s0);
      int i0 = (int)fi;  // tau rounds up to the period at most: row T is row 0
      if (i0 >= d.T) i0 -= d.T;
      s_ri0 = i0;
      s_rf0 = (float)(s0 - fi);
      const float r = d.dt / d.dt_ref;
      s_rr = make_float2(r, fmaf(-r, d.dt_ref, d.dt) / d.dt_ref);
      // rows i0 .. i0 + n - 1 (mod T) hold every step's pair of rows; staged
      // as up to two bulk copies (the second after the wrap to row 0), each
      // from a 16-byte boundary at or below its first row
      const int n = (int)floor((double)s_rf0 + (double)N * ((double)d.dt / (double)d.dt_ref)) + 3;
      s_ref_n1 = 0;
      if (d.ref_rows > 0 && n <= d.ref_rows && n <= d.T) {
        const int n1 = min(n, d.T - i0), n2 = n - n1;
        const uint32_t b0 = 52u * (uint32_t)i0, a0 = b0 & ~15u, len1 = align16(b0 - a0 + 52u * (uint32_t)n1);
        const uint32_t len2 = n2 > 0 ? align16(52u * (uint32_t)n2) : 0u;
        const uint32_t table = 52u * (uint32_t)d.T + (uint32_t)d.ref_pad;
        if (a0 + len1 <= table && len2 <= table && len1 + 16u + len2 <= align16((uint32_t)d.ref_rows * 52u + 16u) + 16u) {
          s_ref_n1 = n1;
          s_ref_lead = (int)(b0 - a0);
          s_ref_seg2 = (int)align16(len1);
          bytes_ref = len1 + len2;
          s_ref_len[0] = len1;
          s_ref_len[1] = len2;
          s_ref_src = a0;
        }
      }
    }
    mbar_expect_tx(&mbar, bytes_U + bytes_path + bytes_gates + bytes_ref);
    bulk_g2s(sU, d.U, bytes_U, &mbar);
    if (bytes_path) bulk_g2s(sPath, d.path, bytes_path, &mbar);
    if (bytes_gates) bulk_g2s(sG, d.gframes, bytes_gates, &mbar);
    if (bytes_ref) {
      bulk_g2s(sRef, reinterpret_cast<const unsigned char*>(d.ref) + s_ref_src, s_ref_len[0], &mbar);
      if (s_ref_len[1]) bulk_g2s(sRef + s_ref_seg2, d.ref, s_ref_len[1], &mbar);
    }
  }
  // GEN != 0: the normals are drawn here (GEN 1 stores them in global memory,
  // GEN 2 draws them again in the epilogue, GEN 3 keeps them in shared
  // memory) instead of being loaded from the noise kernel's output
  const uint32_t iter = GEN ? st->iter : 0u;
  // ---- wait for the bulk copies (bounded) ----
  // A wait that gives up marks the block's samples invalid and counts a
  // timeout, which the solve reports as MPPI_ERR_TIMEOUT; a second bounded
  // wait then lets the copies land before the block uses or releases the
  // shared memory they write.  (For testing, the first wait can target a
  // barrier that no copy ever completes.)
  __syncthreads();
  if (!mbar_wait(d.wait_unreachable ? &mbar_never : &mbar, 0, d.wait_ns)) {
    if (tid == 0) { s_bad = 1; atomicAdd(&st->timeouts, 1); }
    mbar_wait(&mbar, 0, 200000000ull);
  }
  __syncthreads();
  if (OBJ == MPPI_OBJ_GATE) {
    if (tid == 0) {
      // the plant's own pass of the current gate since the last solve
      int adv = 0;
      if (st->has_prev && !(d.closed == 0 && st->gate >= d.n_gates)) {
        const GateF g = load_gate(sG, gate_slot(st->gate, d.n_gates, d.closed));
        const float* p0 = st->prev_x0;
        const float sa = plane_dist(g, p0[0], p0[1]), sb = plane_dist(g, x0s[0], x0s[1]);
        if (sa < 0.f && sb >= 0.f &&
            through_opening(g, sa, sb, p0[0], p0[1], p0[2], x0s[0] - p0[0], x0s[1] - p0[1], x0s[2] - p0[2]))
          adv = 1;
      }
      s_adv = adv;
      s_gate0 = st->gate + adv;
      s_slot0 = gate_slot(st->gate + adv, d.n_gates, d.closed);
    }
    __syncthreads();
    for (int k = tid; k < N; k += blockDim.x) sPrev[k] = max(0, d.prevcnt[k] - s_adv);
  }
  if (OBJ == MPPI_OBJ_TRACK) {
    // reference window x_ref(t0 + k dt), k = 0..N: linear in the table, nlerp
    // for q, from the staged rows (or the table, where they were not staged)
    const float2 rr = s_rr;
    const int n1 = s_ref_n1;
    auto row = [&](int i) -> const float* {
      if (!n1) return d.ref + (size_t)13 * i;
      int q = i - s_ri0;
      if (q < 0) q += d.T;
      return reinterpret_cast<const float*>(q < n1 ? sRef + s_ref_lead + 52 * q : sRef + s_ref_seg2 + 52 * (q - n1));
    };
    for (int k = tid; k <= N; k += blockDim.x) {
      const float kf = (float)k;
      const float p = kf * rr.x;
      const float pe = fmaf(kf, rr.x, -p) + kf * rr.y;
      const float ip = floorf(p);
      float f = ((p - ip) + pe) + s_rf0;
      const float fl = floorf(f);
      f -= fl;
      int i = (s_ri0 + (int)ip + (int)fl) % d.T;
      if (i < 0) i += d.T;
      const int i1 = i + 1 < d.T ? i + 1 : 0;
      const float* a = row(i);
      const float* b = row(i1);
      float* o = sX + (size_t)13 * k;
      float* ol = sXl + (size_t)4 * k;
      for (int c = 0; c < 13; ++c) o[c] = fmaf(f, b[c] - a[c], a[c]);
      // positions as (hi, lo): the error terms are then formed relative to
      // the table row instead of to a binary32 rounding of it
      for (int c = 0; c < 3; ++c) ol[c] = fmaf(f, b[c] - a[c], a[c] - o[c]);
      ol[3] = 0.f;
      const float dot = a[6] * b[6] + a[7] * b[7] + a[8] * b[8] + a[9] * b[9];
      const float sg = dot < 0.f ? -1.f : 1.f;
      float n2 = 0.f;
      for (int c = 6; c < 10; ++c) {
        o[c] = (1.f - f) * a[c] + f * sg * b[c];
        n2 += o[c] * o[c];
      }
      const float rn = 1.0f / sqrtf(n2);
      for (int c = 6; c < 10; ++c) o[c] *= rn;
    }
    __syncthreads();
  }
  if (OBJ == MPPI_OBJ_CONTOUR) {
    // theta_0: closest point of the path to x0 among the node segments of the
    // window [theta_prev - back, theta_prev + ahead] (whole path on the first
    // solve).  The window's node indices come from the FP64 progress state,
    // once per block (one thread; the search itself is binary32).
    if (tid == 0) {
      int jlo = 0, jhi = d.S - 1;
      if (st->has_theta) {
        const double dsd = (double)d.L / (double)d.S;
        jlo = (int)floor((st->theta - (double)d.theta_back) / dsd);
        jhi = (int)floor((st->theta + (double)d.theta_ahead) / dsd);
      }
      s_win[0] = jlo;
      s_win[1] = jhi;
    }
    __syncthreads();
    const int jlo = s_win[0], jhi = s_win[1];
    float best = INFINITY, bt = 0.f;
    int bj = 0x7fffffff;
    for (int jj = jlo + tid; jj <= jhi; jj += blockDim.x) {
      int j = jj % d.S;
      if (j < 0) j += d.S;
      const int j1 = (j + 1) % d.S;
      const float* a = path + 6 * j;
      const float* b = path + 6 * j1;
      const float dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
      const float rx = x0s[0] - a[0], ry = x0s[1] - a[1], rz = x0s[2] - a[2];
      float t = (rx * dx + ry * dy + rz * dz) / (dx * dx + dy * dy + dz * dz);
      t = clampf(t, 0.f, 1.f);
      const float ex = rx - t * dx, ey = ry - t * dy, ez = rz - t * dz;
      const float dist = ex * ex + ey * ey + ez * ez;
      if (dist < best || (dist == best && jj < bj)) { best = dist; bj = jj; bt = t; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      const float ot = __shfl_xor_sync(0xffffffffu, bt, o);
      if (od < best || (od == best && oj < bj)) { best = od; bj = oj; bt = ot; }
    }
    if (lane == 0) { s_best_d[wid] = best; s_best_j[wid] = bj; s_best_t[wid] = bt; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < nw; ++w)
        if (s_best_d[w] < best || (s_best_d[w] == best && s_best_j[w] < bj)) {
          best = s_best_d[w]; bj = s_best_j[w]; bt = s_best_t[w];
        }
      int j = bj % d.S;
      if (j < 0) j += d.S;
      s_j0 = j;
      s_f0 = bt * d.ds;  // metres past node j0
      const double th = ((double)j + (double)bt) * ((double)d.L / (double)d.S);
      s_theta0 = th;
      s_vth0 = st->has_theta ? (float)st->v_theta : 0.f;
    }
    __syncthreads();
  }
  if (tile.m0 == 0 && OBJ == MPPI_OBJ_TRACK) {
    for (int i = tid; i < (N + 1) * kNX; i += blockDim.x) d.xref[i] = sX[i];
  }

  // ---- the rollout: the thread's samples one after another ----
  const bool five = nu == 5;
  ModelRegs M;
  M.inv_mass = d.inv_mass; M.gravity = d.gravity; M.k_omega = d.k_omega;
  M.g0 = d.gyro[0]; M.g1 = d.gyro[1]; M.g2 = d.gyro[2];
  M.d0 = d.drag[0]; M.d1 = d.drag[1]; M.d2 = d.drag[2]; M.has_drag = d.has_drag;
  RotorRegs RR = rotor_regs(d);
#pragma unroll 1
  for (int rep = 0; rep < spt; ++rep) {
    const int m = tile.m0 + tid + rep * B;
    const bool active = tid < B && m < K && !s_bad;
    float Jh = 0.f, Jc = 0.f;
    int passed = 0, first = -1;
    if (active) {
      Quad s;
      quad_init(s, x0s);
      const float h = d.dt;
      // rotor thrusts (rotor model): the controller's integrated commands
      float Tr[4] = {0.f, 0.f, 0.f, 0.f}, Trc[4] = {0.f, 0.f, 0.f, 0.f};
      if (ROT) {
        const bool hr = st->has_rotor != 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) Tr[r] = hr ? st->rotor[r] : 0.25f * d.hover;
      }
      float dT2 = 0.f;
      // objective state
      // gate progress state: p_k - g for the target gate (ra), its plane
      // distance; the target is gate (s_gate0 + passed), where s_gate0, the
      // solve's current gate, and its table row s_slot0 are the block's
      // (shared memory, not registers)
      // the target gate's frame, read from shared memory where it is used
      const GateF* gp = sG;
      float sa = 0.f, rax = 0.f, ray = 0.f, raz = 0.f;
      if (OBJ == MPPI_OBJ_GATE) {
        gp = sG + s_slot0;
        rax = s.px - gp->cx;
        ray = s.py - gp->cy;
        raz = s.pz - gp->cz;
        sa = gp->nx * rax + gp->ny * ray;
      }
      int node = 0;
      float frac_m = 0.f, frac_c = 0.f, vth = 0.f, c_prev = 0.f;
      if (OBJ == MPPI_OBJ_CONTOUR) {
        node = s_j0;
        frac_m = s_f0;
        vth = s_vth0;
        c_prev = st->has_prev ? st->c_last : d.hover;
      }
      // loop invariants in registers (the descriptor lives in shared memory)
      // software pipeline: the next step's noise is in flight during this step
      float z[kNU], zn[kNU];
      const int it = tid + rep * B;  // the sample's place in the tile
      if (GEN)
        gen_noise<BF16, GEN == 1>(d, iter, m, 0, zn, five);
      else
        load_noise<BF16>(d, (size_t)m, zn, five);
      if (GEN == 3) {
        sZ4[it] = make_float4(zn[0], zn[1], zn[2], zn[3]);
        if (five) sZ5[it] = zn[4];
      }
#pragma unroll kRolloutUnroll
      for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int j = 0; j < kNU; ++j) z[j] = zn[j];
        if (k + 1 < N) {
          if (GEN)
            gen_noise<BF16, GEN == 1>(d, iter, m, k + 1, zn, five);
          else
            load_noise<BF16>(d, (size_t)(k + 1) * K + m, zn, five);
          if (GEN == 3) {
            sZ4[(size_t)(k + 1) * TS + it] = make_float4(zn[0], zn[1], zn[2], zn[3]);
            if (five) sZ5[(size_t)(k + 1) * TS + it] = zn[4];
          }
        }
        const float* Uk = sU + kNU * k;
        // sampling (Eq. 3 with the clamp): sigma and the input bounds are
        // read from shared memory every step rather than held in 12
        // registers (the rollout is built for 96 registers; held, they
        // pushed the gate-progress rollout into spills)
        const float4 b0 = lds4_volatile(sBnd), b1 = lds4_volatile(sBnd + 1), b2 = lds4_volatile(sBnd + 2),
                     b3 = lds4_volatile(sBnd + 3);
        const float u0 = clampf(Uk[0] + b0.x * z[0], b0.y, b0.z);
        const float u1 = clampf(Uk[1] + b1.x * z[1], b1.y, b1.z);
        const float u2 = clampf(Uk[2] + b2.x * z[2], b2.y, b2.z);
        const float u3 = clampf(Uk[3] + b3.x * z[3], b3.y, b3.z);
        float stage = 0.f;
        if (OBJ == MPPI_OBJ_TRACK) {
          // Eq. 8 stage term on x_k and u_k
          const float* xr = sX + kNX * k;
          const float* xl = sXl + 4 * k;
          const float dot = s.qw * xr[6] + s.qx * xr[7] + s.qy * xr[8] + s.qz * xr[9];
          const float sg = dot < 0.f ? -1.f : 1.f;
          float e;
          e = ((s.px - xr[0]) - s.cpx) - xl[0]; stage += d.Q[0] * e * e;
          e = ((s.py - xr[1]) - s.cpy) - xl[1]; stage += d.Q[1] * e * e;
          e = ((s.pz - xr[2]) - s.cpz) - xl[2]; stage += d.Q[2] * e * e;
          e = (s.vx - xr[3]) - s.cvx; stage += d.Q[3] * e * e;
          e = (s.vy - xr[4]) - s.cvy; stage += d.Q[4] * e * e;
          e = (s.vz - xr[5]) - s.cvz; stage += d.Q[5] * e * e;
          e = (s.qw - sg * xr[6]) - s.cqw; stage += d.Q[6] * e * e;
          e = (s.qx - sg * xr[7]) - s.cqx; stage += d.Q[7] * e * e;
          e = (s.qy - sg * xr[8]) - s.cqy; stage += d.Q[8] * e * e;
          e = (s.qz - sg * xr[9]) - s.cqz; stage += d.Q[9] * e * e;
          e = s.wx - xr[10]; stage += d.Q[10] * e * e;
          e = s.wy - xr[11]; stage += d.Q[11] * e * e;
          e = s.wz - xr[12]; stage += d.Q[12] * e * e;
          const float du = ROT ? u0 : u0 - d.hover;  // rotor model: the rates themselves
          stage += d.R[0] * du * du + d.R[1] * u1 * u1 + d.R[2] * u2 * u2 + d.R[3] * u3 * u3;
        }
        float near = 0.f;
        if (OBJ == MPPI_OBJ_GATE) {
          // Eq. 7 near-gate term on p_k and the solve's current gate g0
          float ex = rax, ey = ray, ez = raz;
          if (passed) {
            const GateF& G0 = sG[s_slot0];
            ex = (s.px - G0.cx) - s.cpx;
            ey = (s.py - G0.cy) - s.cpy;
            ez = (s.pz - G0.cz) - s.cpz;
          }
          const float d0 = ex * ex + ey * ey + ez * ez;
          const float4 nr = lds4_volatile(sBnd + 5);  // (q_near, r_near^2): read here, not held
          near = d0 < nr.y ? nr.x * d0 : 0.f;
        }
        float dpx, dpy, dpz;
        if (ROT) {
          if (M.has_drag)
            rk4_step_rotor<true>(M, RR, &d.stepc, s, k ? 0.f : s_qe0, Tr, Trc, u0, u1, u2, u3, h, dpx, dpy, dpz, dT2);
          else
            rk4_step_rotor<false>(M, RR, &d.stepc, s, k ? 0.f : s_qe0, Tr, Trc, u0, u1, u2, u3, h, dpx, dpy, dpz, dT2);
        } else {
          if (M.has_drag)
            rk4_step<true>(M, &d.stepc, s, k ? 0.f : s_qe0, u0, u1, u2, u3, h, dpx, dpy, dpz);
          else
            rk4_step<false>(M, &d.stepc, s, k ? 0.f : s_qe0, u0, u1, u2, u3, h, dpx, dpy, dpz);
        }
        if (OBJ == MPPI_OBJ_GATE) {
          // Eq. 7: ||p_{k+1} - g||^2 - ||p_k - g||^2 = (p_{k+1} - p_k) . (p_{k+1} + p_k - 2 g),
          // with both positions taken relative to g before rounding
          float rbx = (s.px - gp->cx) - s.cpx, rby = (s.py - gp->cy) - s.cpy, rbz = (s.pz - gp->cz) - s.cpz;
          stage = dpx * (rax + rbx) + dpy * (ray + rby) + dpz * (raz + rbz) + near;
          float sb = gp->nx * rbx + gp->ny * rby;
          if (sa < 0.f && sb >= 0.f) {
            const bool open_track_done = (d.closed == 0) && s_gate0 + passed >= d.n_gates;
            const bool ok_time = d.temporal_rule == MPPI_RULE_OFF || sPrev[k] <= passed;
            // crossing point on the segment, relative to the gate centre
            const float a = sa / (sa - sb);
            const float ex = rax + a * (rbx - rax), ey = ray + a * (rby - ray), ez = raz + a * (rbz - raz);
            const bool open = fabsf(-gp->ny * ex + gp->nx * ey) <= gp->hw && fabsf(ez) <= gp->hh;
            if (!open_track_done && ok_time && open) {
              ++passed;
              if (first < 0) first = k;
              gp = sG + gate_slot(s_gate0 + passed, d.n_gates, d.closed);
              rbx = (s.px - gp->cx) - s.cpx;
              rby = (s.py - gp->cy) - s.cpy;
              rbz = (s.pz - gp->cz) - s.cpz;
              sb = gp->nx * rbx + gp->ny * rby;
            }
          }
          rax = rbx;
          ray = rby;
          raz = rbz;
          sa = sb;
        } else if (OBJ == MPPI_OBJ_CONTOUR) {
          // Eq. 9 with the progress state (theta, v_theta), terms on x_{k+1}
          const float a = clampf(Uk[4] + d.sigma[4] * z[4], d.u_min[4], d.u_max[4]);
          const float v1 = clampf(vth + a * h, 0.f, d.v_theta_max);
          kahan_add(frac_m, frac_c, 0.5f * (vth + v1) * h);
          float fm = frac_m - frac_c;
          while (fm >= d.ds) {
            frac_m -= d.ds;
            fm = frac_m - frac_c;
            if (++node >= d.S) node -= d.S;
          }
          const float fr = fm * d.inv_ds;
          const int n1 = node + 1 >= d.S ? 0 : node + 1;
          const float* A = path + 6 * node;
          const float* Bn = path + 6 * n1;
          // e = p - P(theta) with P = A + fr (B - A), formed as (p - A) - fr (B - A)
          float Tx = A[3] + fr * (Bn[3] - A[3]), Ty = A[4] + fr * (Bn[4] - A[4]), Tz = A[5] + fr * (Bn[5] - A[5]);
          const float rn = rsqrtf(Tx * Tx + Ty * Ty + Tz * Tz);
          Tx *= rn; Ty *= rn; Tz *= rn;
          const float ex = ((s.px - A[0]) - fr * (Bn[0] - A[0])) - s.cpx;
          const float ey = ((s.py - A[1]) - fr * (Bn[1] - A[1])) - s.cpy;
          const float ez = ((s.pz - A[2]) - fr * (Bn[2] - A[2])) - s.cpz;
          const float et = ex * Tx + ey * Ty + ez * Tz;
          const float cx = ex - et * Tx, cy = ey - et * Ty, cz = ez - et * Tz;
          // thrust change: the collective command, or the rotor thrusts (rotor model)
          const float dT = u0 - c_prev;
          const float dTT = ROT ? dT2 : dT * dT;
          stage = d.q_lag * et * et + d.q_cont * (cx * cx + cy * cy + cz * cz) +
                  d.q_omega[0] * s.wx * s.wx + d.q_omega[1] * s.wy * s.wy + d.q_omega[2] * s.wz * s.wz +
                  d.r_dv * a * a + d.r_dthrust * dTT - d.mu * v1;
          c_prev = u0;
          vth = v1;
        } else {
          if (k == N - 1) {
            const float* xr = sX + kNX * N;
            const float* xl = sXl + 4 * N;
            const float dot = s.qw * xr[6] + s.qx * xr[7] + s.qy * xr[8] + s.qz * xr[9];
            const float sg = dot < 0.f ? -1.f : 1.f;
            float e;
            e = ((s.px - xr[0]) - s.cpx) - xl[0]; stage += d.QN[0] * e * e;
            e = ((s.py - xr[1]) - s.cpy) - xl[1]; stage += d.QN[1] * e * e;
            e = ((s.pz - xr[2]) - s.cpz) - xl[2]; stage += d.QN[2] * e * e;
            e = (s.vx - xr[3]) - s.cvx; stage += d.QN[3] * e * e;
            e = (s.vy - xr[4]) - s.cvy; stage += d.QN[4] * e * e;
            e = (s.vz - xr[5]) - s.cvz; stage += d.QN[5] * e * e;
            e = (s.qw - sg * xr[6]) - s.cqw; stage += d.QN[6] * e * e;
            e = (s.qx - sg * xr[7]) - s.cqx; stage += d.QN[7] * e * e;
            e = (s.qy - sg * xr[8]) - s.cqy; stage += d.QN[8] * e * e;
            e = (s.qz - sg * xr[9]) - s.cqz; stage += d.QN[9] * e * e;
            e = s.wx - xr[10]; stage += d.QN[10] * e * e;
            e = s.wy - xr[11]; stage += d.QN[11] * e * e;
            e = s.wz - xr[12]; stage += d.QN[12] * e * e;
          }
        }
        {
          const float4 bl = lds4_volatile(sBnd + 4);
          stage += limit_penalty(bl.x, bl.y, bl.z, s);
        }
        kahan_add(Jh, Jc, stage);
      }
    }

    // per-sample outputs; the cost pair stays in shared memory for Eq. 4
    const bool valid = active && isfinite(Jh) && isfinite(Jc) && isfinite(Jh - Jc);
    if (active) {
      d.J[m] = pack2(Jh, -Jc);  // the compensated pair itself: no FP64 arithmetic here
      d.info[m] = passed | ((first + 1) << 16);
    }
    if (tid < B) {
      sJ[tid + rep * B] = valid ? Jh : NAN;
      sJ[TS + tid + rep * B] = Jc;
    }
  }  // samples of this thread

  // ---- the block's share of Eq. 4 ----
  const int acc = d.accum;
  // (with GEN 1 the epilogue reads noise other threads of this block stored;
  // the barriers inside the block reductions make those stores visible)
  double m_t, S_t;  // tile minimum and sum of exp weights (packed (hi, lo) unless FP64)
  const int own = tid < B ? spt : 0;  // this thread's entries of sJ / sE
  if (acc == MPPI_ACC_F64) {
    double mloc = INFINITY;
    for (int r = 0; r < own; ++r) {
      const int i = tid + r * B;
      if (isfinite(sJ[i])) mloc = fmin(mloc, (double)sJ[i] - (double)sJ[TS + i]);
    }
    m_t = block_min_d(mloc, red);
    double se = 0.0;
    for (int r = 0; r < own; ++r) {
      const int i = tid + r * B;
      float e = 0.f;
      if (isfinite(sJ[i]) && !isinf(m_t))
        e = expf(-(float)(((double)sJ[i] - (double)sJ[TS + i]) - m_t) * d.inv_lambda);
      sE[i] = e;
      se += (double)e;
    }
    S_t = block_sum_d(se, red);  // also publishes sE
  } else {
    // any common shift leaves Eq. 4 unchanged: the binary32 minimum of the
    // rounded costs serves; J - m_t is formed from the compensated pair
    float* redf = reinterpret_cast<float*>(red);
    float mloc = INFINITY;
    for (int r = 0; r < own; ++r) {
      const int i = tid + r * B;
      if (isfinite(sJ[i])) mloc = fminf(mloc, sJ[i] - sJ[TS + i]);
    }
    const float mf = block_min_f(mloc, redf);
    float sh = 0.f, sl = 0.f;
    for (int r = 0; r < own; ++r) {
      const int i = tid + r * B;
      float e = 0.f;
      if (isfinite(sJ[i]) && !isinf(mf)) e = expf(-(((sJ[i] - mf) - sJ[TS + i]) * d.inv_lambda));
      sE[i] = e;
      if (r == 0)
        sh = e;
      else
        add2(sh, sl, e, 0.f);
    }
    block_sum2_f(sh, sl, redf);  // also publishes sE
    m_t = (double)mf;
    S_t = pack2(sh, sl);
  }

  // ---- weighted deviation sums per (step, input) of this tile (Eq. 5) ----
  const int nvalid = min(TS, K - tile.m0);
  const int NNU = N * kNU;
  const int tile_in_solve = tile.m0 / TS;
  double* myP = d.part_P + (size_t)tile_in_solve * NNU;
  switch (acc) {
    case MPPI_ACC_F64: eq5_rows<MPPI_ACC_F64, BF16, GEN>(d, sU, sE, iter, tile.m0, nvalid, myP, sZ4, sZ5, TS); break;
    case MPPI_ACC_F32: eq5_rows<MPPI_ACC_F32, BF16, GEN>(d, sU, sE, iter, tile.m0, nvalid, myP, sZ4, sZ5, TS); break;
    default: eq5_rows<MPPI_ACC_KAHAN32, BF16, GEN>(d, sU, sE, iter, tile.m0, nvalid, myP, sZ4, sZ5, TS); break;
  }
  if (tid == 0) {
    d.part_m[tile_in_solve] = m_t;
    d.part_S[tile_in_solve] = S_t;
  }

  // ---- two-level merge: last block of each group, then last group ----
  constexpr int kMergePre = (GEN == 0 && ROT == 0) ? 8 : 0;
  const int T = d.n_tiles;
  const int G = group_size_for(T);
  const int n_groups = (T + G - 1) / G;
  const int grp = tile_in_solve / G;
  const int gsize = min(G, T - grp * G);
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const uint32_t c = atomicAdd(d.ticket + 1 + grp, 1u);
    s_group_last = (c == (uint32_t)gsize - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_group_last) return;
  __threadfence();
  const int f64 = acc == MPPI_ACC_F64;
  double* gm = d.part_m + T;
  double* gS = d.part_S + T;
  double* gP = d.part_P + (size_t)T * NNU;
  if (n_groups > 1) {
    MergeIn in{d.part_m + grp * G, d.part_S + grp * G, d.part_P + (size_t)grp * G * NNU};
    merge_partials<kMergePre>(d, in, gsize, NNU, gm + grp, gS + grp, gP + (size_t)grp * NNU, sMerge, red, f64);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      d.ticket[1 + grp] = 0u;
      const uint32_t c = atomicAdd(d.ticket, 1u);
      s_last = (c == (uint32_t)n_groups - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
  } else if (tid == 0) {
    d.ticket[1 + grp] = 0u;
  }
  // final merge -> U*_new = U* + P / S
  {
    // timeouts counted by any block of this solve: each block counts before
    // its ticket, so the count is complete here; requested now, used at the end
    const int32_t timeouts = tid == 0 ? *reinterpret_cast<volatile const int32_t*>(&st->timeouts) : 0;
    MergeIn in;
    int n;
    if (n_groups > 1) {
      in = MergeIn{gm, gS, gP};
      n = n_groups;
    } else {
      in = MergeIn{d.part_m, d.part_S, d.part_P};
      n = T;
    }
    // the final sums stay in shared memory
    double* fP = reinterpret_cast<double*>(smem + Ls.off_fin);
    merge_partials<kMergePre>(d, in, n, NNU, &s_m, &s_S, fP, sMerge, red, f64);
    __threadfence_block();
    __syncthreads();
    const float2 S2 = unpack2(s_S);
    const double S_total = f64 ? s_S : (double)S2.x + (double)S2.y;
    const bool degenerate = isinf(s_m) || !(S_total > 0.0);
    float* u0o = io.u0 + (size_t)tile.solve * kNU;
    for (int o = tid; o < NNU; o += blockDim.x) {
      const int k = o / kNU, j = o - k * kNU;
      float v = sU[o];
      if (!degenerate && j < nu) {
        if (f64) {
          v = (float)((double)sU[o] + fP[o] / s_S);
        } else {
          // (P_hi + P_lo) / (S_hi + S_lo) with one correction step
          const float2 P2 = unpack2(fP[o]);
          float q = P2.x / S2.x;
          const float r = (fmaf(-q, S2.x, P2.x) + P2.y) - q * S2.y;
          q += r / S2.x;
          v = sU[o] + q;
        }
      }
      if (j >= nu) v = 0.f;
      d.unew[o] = v;
      sU[o] = v;  // U*_new replaces U* here (each entry is this thread's own)
      if (k == 0) u0o[j] = v;
    }
    __syncthreads();
    // warm start: shift by one (or keep the sequence), repeat the last row
    // over the whole capacity
    const int shift = d.warm_keep ? 0 : 1;
    for (int o = tid; o < d.N_cap * kNU; o += blockDim.x) {
      const int k = o / kNU, j = o - k * kNU;
      const int src = min(k + shift, N - 1);
      d.U[o] = sU[src * kNU + j];
    }
    if (tid < kNX) st->prev_x0[tid] = x0s[tid];
    if (tid == 0) {
      const float c0 = sU[0];
      st->gate0 = st->gate + (OBJ == MPPI_OBJ_GATE ? s_adv : 0);
      st->adv = OBJ == MPPI_OBJ_GATE ? s_adv : 0;
      st->gate = st->gate0;
      const int32_t to = timeouts;
      const int status = to != st->timeouts_seen ? MPPI_ERR_TIMEOUT : degenerate ? MPPI_WARN_DEGENERATE : MPPI_OK;
      st->timeouts_seen = to;
      st->status = status;
      st->iter += 1u;
      st->has_prev = 1;
      st->n_nom = N;
      st->c_last = c0;
      if (ROT) {
        // the plant applies u0 (rotor-thrust rates) for one control period
        const bool hr = st->has_rotor != 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float t0r = hr ? st->rotor[r] : 0.25f * d.hover;
          st->rotor_prev[r] = t0r;
          st->rotor[r] = clampf(t0r + sU[r] * d.dt, d.thrust_min, d.thrust_max);
        }
        st->has_rotor = 1;
      }
      if (OBJ == MPPI_OBJ_CONTOUR) {
        const float a0 = sU[4];
        st->theta = s_theta0;
        st->v_theta = (double)clampf(s_vth0 + a0 * d.dt, 0.f, d.v_theta_max);
        st->has_theta = 1;
        st->scal[0] = s_theta0;
        st->scal[1] = (double)s_vth0;
      }
      st->scal[2] = s_m;
      st->scal[3] = S_total;
      if (io.status) io.status[tile.solve] = status;
      d.ticket[0] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// per-objective launch and set-up (instantiated in mppi_rollout_<obj>.cu)
// ---------------------------------------------------------------------------
template <int OBJ, int BF16, int ROT>
cudaError_t configure_rollout_t() {
  cudaError_t e = cudaFuncSetAttribute(rollout_kernel<OBJ, BF16, 0, ROT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_kernel<OBJ, BF16, 1, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
  // drawing the noise again in the epilogue stores nothing, so it has no
  // bfloat16 form
  if constexpr (!BF16)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(rollout_kernel<OBJ, 0, 2, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_kernel<OBJ, BF16, 3, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
  return e;
}

template <int OBJ>
cudaError_t configure_rollout_obj() {
  cudaError_t e = configure_rollout_t<OBJ, 0, 0>();
  if (e == cudaSuccess) e = configure_rollout_t<OBJ, 1, 0>();
  // the rotor model is built with float32 noise storage only
  if (e == cudaSuccess) e = configure_rollout_t<OBJ, 0, 1>();
  return e;
}

template <int OBJ, int BF16, int ROT>
cudaError_t launch_rollout_t(const SolveDesc* descs, const Tile* tiles, int n_tiles, int block, uint32_t smem,
                             LaunchIO io, cudaStream_t s, int gen) {
  (void)cudaGetLastError();
  if (gen == 3) {
    rollout_kernel<OBJ, BF16, 3, ROT><<<n_tiles, block, smem, s>>>(descs, tiles, io);
  } else if (gen == 2) {
    if constexpr (BF16) return cudaErrorInvalidValue;
    else rollout_kernel<OBJ, 0, 2, ROT><<<n_tiles, block, smem, s>>>(descs, tiles, io);
  } else if (gen == 1) {
    rollout_kernel<OBJ, BF16, 1, ROT><<<n_tiles, block, smem, s>>>(descs, tiles, io);
  } else {
    rollout_kernel<OBJ, BF16, 0, ROT><<<n_tiles, block, smem, s>>>(descs, tiles, io);
  }
  add_launches(1);
  return cudaGetLastError();
}

template <int OBJ>
cudaError_t launch_rollout_obj(int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles, int block,
                               uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor) {
  if (rotor) {
    if (bf16) return cudaErrorInvalidValue;
    return launch_rollout_t<OBJ, 0, 1>(descs, tiles, n_tiles, block, smem, io, s, gen);
  }
  return bf16 ? launch_rollout_t<OBJ, 1, 0>(descs, tiles, n_tiles, block, smem, io, s, gen)
              : launch_rollout_t<OBJ, 0, 0>(descs, tiles, n_tiles, block, smem, io, s, gen);
}

}  // namespace mppi
