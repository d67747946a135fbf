// FP32 storage and arithmetic instantiations of the step kernel, with the
// displacement accumulated in FP32 or FP64.
#include "lbm_kernels.cuh"
#include "step_fused.cuh"
#include "step2_lam.cuh"

namespace lbm {

template <class U>
static void launch_u(const StepParams &p, bool lam, int mode, dim3 grid, dim3 block,
                     cudaStream_t s) {
  if (mode == 0) {
    if (lam) launch_pdl(step_kernel<float, float, U, true, 0>, grid, block, s, p);
    else launch_pdl(step_kernel<float, float, U, false, 0>, grid, block, s, p);
  } else {
    if (lam) step_kernel<float, float, U, true, 1><<<grid, block, 0, s>>>(p);
    else step_kernel<float, float, U, false, 1><<<grid, block, 0, s>>>(p);
  }
}

void launch_step_f32(const StepParams &p, bool lam, bool u64, int mode, dim3 grid, dim3 block,
                     cudaStream_t s) {
  if (u64) launch_u<double>(p, lam, mode, grid, block, s);
  else launch_u<float>(p, lam, mode, grid, block, s);
}

void launch_step2_f32(const StepParams &p, bool u64, cudaStream_t s) {
  const dim3 grid = step2_grid(p.nx, p.ny), block = step2_block();
  if (u64) launch_pdl(step2_kernel<float, float, double>, grid, block, s, p);
  else launch_pdl(step2_kernel<float, float, float>, grid, block, s, p);
}

void launch_step2_lam_f32(const StepParams &p, bool u64, cudaStream_t s) {
  const dim3 grid = step2_lam_grid(p.nx, p.ny), block = step2_lam_block();
  if (u64) launch_pdl(step2_lam_kernel<float, float, double>, grid, block, s, p);
  else launch_pdl(step2_lam_kernel<float, float, float>, grid, block, s, p);
}

}  // namespace lbm
