// 16-bit population storage (FP16 or BF16) with FP32 arithmetic; the
// displacement is accumulated in FP32 or FP64.
#include "lbm_kernels.cuh"
#include "step_fused.cuh"
#include "step2_lam.cuh"

namespace lbm {

template <class T, class U>
static void launch_tu(const StepParams &p, bool lam, int mode, dim3 grid, dim3 block,
                      cudaStream_t s) {
  if (mode == 0) {
    if (lam) launch_pdl(step_kernel<T, float, U, true, 0>, grid, block, s, p);
    else launch_pdl(step_kernel<T, float, U, false, 0>, grid, block, s, p);
  } else {
    if (lam) step_kernel<T, float, U, true, 1><<<grid, block, 0, s>>>(p);
    else step_kernel<T, float, U, false, 1><<<grid, block, 0, s>>>(p);
  }
}

void launch_step_16(const StepParams &p, bool bf16, bool lam, bool u64, int mode, dim3 grid,
                    dim3 block, cudaStream_t s) {
  if (bf16) {
    if (u64) launch_tu<__nv_bfloat16, double>(p, lam, mode, grid, block, s);
    else launch_tu<__nv_bfloat16, float>(p, lam, mode, grid, block, s);
  } else {
    if (u64) launch_tu<__half, double>(p, lam, mode, grid, block, s);
    else launch_tu<__half, float>(p, lam, mode, grid, block, s);
  }
}

template <class T, class U>
static void launch2(const StepParams &p, cudaStream_t s) {
  launch_pdl(step2_kernel<T, float, U>, step2_grid(p.nx, p.ny), step2_block(), s, p);
}

template <class T, class U>
static void launch2l(const StepParams &p, cudaStream_t s) {
  launch_pdl(step2_lam_kernel<T, float, U>, step2_lam_grid(p.nx, p.ny), step2_lam_block(), s, p);
}

void launch_step2_lam_16(const StepParams &p, bool bf16, bool u64, cudaStream_t s) {
  if (bf16) {
    if (u64) launch2l<__nv_bfloat16, double>(p, s);
    else launch2l<__nv_bfloat16, float>(p, s);
  } else {
    if (u64) launch2l<__half, double>(p, s);
    else launch2l<__half, float>(p, s);
  }
}

void launch_step2_16(const StepParams &p, bool bf16, bool u64, cudaStream_t s) {
  if (bf16) {
    if (u64) launch2<__nv_bfloat16, double>(p, s);
    else launch2<__nv_bfloat16, float>(p, s);
  } else {
    if (u64) launch2<__half, double>(p, s);
    else launch2<__half, float>(p, s);
  }
}

}  // namespace lbm
