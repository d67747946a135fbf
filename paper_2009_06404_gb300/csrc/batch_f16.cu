// Batched step, FP16 or BF16 populations with FP32 arithmetic (FP32 or FP64
// displacement).
#include "batch_kernels.cuh"

namespace lbm {

cudaError_t batch_launch_16(bool bf16, bool u64, int R, int tps, bool persistent,
                            const BatchArgs &a, int count, int grid, bool pdl, cudaStream_t s) {
  if (bf16) {
    if (u64)
      return batch_launch_r<__nv_bfloat16, float, double>(R, tps, persistent, a, count, grid,
                                                          pdl, s);
    return batch_launch_r<__nv_bfloat16, float, float>(R, tps, persistent, a, count, grid, pdl,
                                                       s);
  }
  if (u64)
    return batch_launch_r<__half, float, double>(R, tps, persistent, a, count, grid, pdl, s);
  return batch_launch_r<__half, float, float>(R, tps, persistent, a, count, grid, pdl, s);
}

int batch_occupancy_16(bool bf16, bool u64, int R, int tps) {
  if (bf16)
    return u64 ? batch_occupancy_r<__nv_bfloat16, float, double>(R, tps)
               : batch_occupancy_r<__nv_bfloat16, float, float>(R, tps);
  return u64 ? batch_occupancy_r<__half, float, double>(R, tps)
             : batch_occupancy_r<__half, float, float>(R, tps);
}

}  // namespace lbm
