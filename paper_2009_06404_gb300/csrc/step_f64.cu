// FP64 storage and arithmetic instantiations of the step kernel.
#include "lbm_kernels.cuh"
#include "step_fused.cuh"
#include "step2_lam.cuh"

namespace lbm {

void launch_step_f64(const StepParams &p, bool lam, int mode, dim3 grid, dim3 block,
                     cudaStream_t s) {
  if (mode == 0) {
    if (lam) launch_pdl(step_kernel<double, double, double, true, 0>, grid, block, s, p);
    else launch_pdl(step_kernel<double, double, double, false, 0>, grid, block, s, p);
  } else {
    if (lam) step_kernel<double, double, double, true, 1><<<grid, block, 0, s>>>(p);
    else step_kernel<double, double, double, false, 1><<<grid, block, 0, s>>>(p);
  }
}

void launch_step2_f64(const StepParams &p, cudaStream_t s) {
  launch_pdl(step2_kernel<double, double, double>, step2_grid(p.nx, p.ny), step2_block(), s, p);
}

void launch_step2_lam_f64(const StepParams &p, cudaStream_t s) {
  launch_pdl(step2_lam_kernel<double, double, double>, step2_lam_grid(p.nx, p.ny),
             step2_lam_block(), s, p);
}

}  // namespace lbm
