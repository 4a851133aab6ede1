// mppi_launch.h -- host-side entry points of the kernels (internal to libmppi)
#pragma once
#include <cuda_runtime.h>

#include "mppi_device.cuh"

namespace mppi {

// partials of a solve are merged in groups of this size (two-level tree);
// T <= 16 tiles merge in one level
__host__ __device__ inline int group_size_for(int T) {
  if (T <= 16) return T;
  int g = 1;
  while (g * g < T) ++g;
  return g < 8 ? 8 : g;
}
__host__ __device__ inline int n_groups_for(int T) {
  const int G = group_size_for(T);
  return (T + G - 1) / G;
}

__host__ __device__ int path_fits_smem(int S);
// dynamic shared memory of a rollout launch (gen: MPPI_NOISEGEN_*)
uint32_t rollout_smem_bytes(int N, int objective, int S, int block, int merge_cap, int gen, int ref_rows);
// reference rows a tracking block stages in shared memory for a horizon of
// N_cap steps (0: the window reads the table in global memory)
inline int ref_rows_for(int N_cap, float dt, float dt_ref, int T) {
  if (!(dt_ref > 0.f) || T < 2) return 0;
  const double rows = (double)N_cap * (double)dt / (double)dt_ref + 4.0;
  return rows * 52.0 <= 48.0 * 1024.0 && rows <= (double)T ? (int)rows : 0;
}
// frames of n gates from the [n][6] table (device pointers)
cudaError_t launch_gate_frames(const float* raw, int n, GateF* out, cudaStream_t s);
// largest dynamic shared memory a rollout launch may use
constexpr uint32_t kRolloutSmemMax = 200 * 1024;
unsigned long long launches_so_far();
void add_launches(int n);  // kernels run by a graph launch
// model, sampling and cost fields of a descriptor from the C-ABI structs
void fill_model_params(const mppi_model_t& m, const mppi_params_t& p, int nu, SolveDesc& d);
// the (hi, lo) step constants and rotor torque factors of a descriptor
void fill_step_consts(const mppi_model_t& m, float dt, SolveDesc& d);
// records the message mppi_last_error() returns on this thread
void set_last_error(const char* msg);
// sets the dynamic shared-memory limit of every rollout kernel (once per device)
cudaError_t configure_kernels();
// largest block the rollout kernel was compiled for
int rollout_max_block();

// nominal: every solve of the launch has nominal_sample set (sample 0 is stored as zeros);
// N_max: the longest horizon among the launch's solves (a launch of few tiles
// is split along the horizon)
cudaError_t launch_noise(const SolveDesc* descs, const Tile* tiles, int n_tiles, int block, int bf16,
                         cudaStream_t s, int nominal, int N_max);
cudaError_t launch_rollout(int objective, int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles,
                           int block, uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor);
cudaError_t launch_nominal(const SolveDesc* descs, const int32_t* which, int n, cudaStream_t s);
// the rollout kernel's instances, one translation unit per objective
cudaError_t configure_rollout_gate();
cudaError_t configure_rollout_contour();
cudaError_t configure_rollout_track();
cudaError_t launch_rollout_gate(int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles, int block,
                                uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor);
cudaError_t launch_rollout_contour(int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles, int block,
                                   uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor);
cudaError_t launch_rollout_track(int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles, int block,
                                 uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                          uint32_t* out, cudaStream_t s);
cudaError_t launch_normals(uint32_t seed, uint32_t drone, uint32_t k, uint32_t it, uint32_t blk, int n, float* out,
                           cudaStream_t s);
cudaError_t launch_rollout_states(const SolveDesc& md, float dt, int N, int B, const float* x0, const float* U,
                                  float* X, cudaStream_t s, const float* T0, float* Tout);

}  // namespace mppi
