// Batched step, FP64 populations and displacement.
#include "batch_kernels.cuh"

namespace lbm {

cudaError_t batch_launch_f64(int R, int cpt, bool persistent, const BatchArgs &a, int count,
                             int grid, bool pdl, cudaStream_t s) {
  return batch_launch_r<double, double, double>(R, cpt, persistent, a, count, grid, pdl, s);
}

int batch_occupancy_f64(int R, int cpt) {
  return batch_occupancy_r<double, double, double>(R, cpt);
}

}  // namespace lbm
