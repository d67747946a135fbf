// Adjoint step, FP32 compute type.
#include "adjoint_kernels.cuh"

namespace lbm {

cudaError_t adj_step_f32(const AdjParams &a, cudaStream_t s) { return adj_step_t<float>(a, s); }

cudaError_t adj_inject_f32(void *ubar_r, void *jrec, const int *rec_id, int nrec,
                           const double *d, cudaStream_t s) {
  return adj_inject_t<float>(ubar_r, jrec, rec_id, nrec, d, s);
}

}  // namespace lbm
