// Batched step, FP32 populations (FP32 or FP64 displacement).
#include "batch_kernels.cuh"

namespace lbm {

cudaError_t batch_launch_f32(bool u64, int R, int tps, bool persistent, const BatchArgs &a,
                             int count, int grid, bool pdl, cudaStream_t s) {
  if (u64) return batch_launch_r<float, float, double>(R, tps, persistent, a, count, grid, pdl, s);
  return batch_launch_r<float, float, float>(R, tps, persistent, a, count, grid, pdl, s);
}

int batch_occupancy_f32(bool u64, int R, int tps) {
  return u64 ? batch_occupancy_r<float, float, double>(R, tps)
             : batch_occupancy_r<float, float, float>(R, tps);
}

__global__ void batch_advance_kernel(BatchHdr *h, int g) { h->kbase += g; }

}  // namespace lbm
