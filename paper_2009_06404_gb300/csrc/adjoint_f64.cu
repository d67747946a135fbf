// Adjoint step, FP64 compute type.
#include "adjoint_kernels.cuh"

namespace lbm {

cudaError_t adj_step_f64(const AdjParams &a, cudaStream_t s) { return adj_step_t<double>(a, s); }

cudaError_t adj_inject_f64(void *ubar_r, void *jrec, const int *rec_id, int nrec,
                           const double *d, cudaStream_t s) {
  return adj_inject_t<double>(ubar_r, jrec, rec_id, nrec, d, s);
}

}  // namespace lbm
