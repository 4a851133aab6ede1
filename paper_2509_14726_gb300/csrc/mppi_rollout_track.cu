// mppi_rollout_track.cu -- the rollout kernel's instances for the track
// objective (see mppi_rollout.cuh); one translation unit per objective so that
// they compile in parallel.
#include "mppi_rollout.cuh"

namespace mppi {

cudaError_t configure_rollout_track() { return configure_rollout_obj<MPPI_OBJ_TRACK>(); }

cudaError_t launch_rollout_track(int bf16, const SolveDesc* descs, const Tile* tiles, int n_tiles, int block,
                              uint32_t smem, LaunchIO io, cudaStream_t s, int gen, int rotor) {
  return launch_rollout_obj<MPPI_OBJ_TRACK>(bf16, descs, tiles, n_tiles, block, smem, io, s, gen, rotor);
}

}  // namespace mppi
