// Adjoint step, FP64 compute type.
#include "adjoint_kernels.cuh"

namespace lbm {

cudaError_t adj_step_f64(const AdjParams &a, bool fused, cudaStream_t s) {
  return adj_step_t<double>(a, fused, s);
}

cudaError_t adj_jrec_f64(const double *d, const int *rec_id, int nrec, int T, void *jrec,
                         cudaStream_t s) {
  return adj_jrec_t<double>(d, rec_id, nrec, T, jrec, s);
}

}  // namespace lbm
