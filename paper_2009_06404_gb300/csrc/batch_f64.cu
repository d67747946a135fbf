// Batched step, FP64 populations and displacement.
#include "batch_kernels.cuh"

namespace lbm {

cudaError_t batch_launch_f64(int R, int tps, bool persistent, const BatchArgs &a, int count,
                             int grid, bool pdl, cudaStream_t s) {
  return batch_launch_r<double, double, double>(R, tps, persistent, a, count, grid, pdl, s);
}

int batch_occupancy_f64(int R, int tps) {
  return batch_occupancy_r<double, double, double>(R, tps);
}

}  // namespace lbm
