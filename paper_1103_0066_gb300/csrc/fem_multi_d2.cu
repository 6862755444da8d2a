// Multi-mesh forward, adjoint element pass and vertex reduction on triangles
// (kernels in fem_multi.cuh).
#include "fem_multi.cuh"

namespace fem {

cudaError_t launch_fwd_multi_d2(int form, const FwdMulti& P, cudaStream_t st) {
  switch (form) {
    case LAPLACE_P1: return launch_fwd_multi_t<2, LAPLACE_P1, JAC_COMP>(P, st);
    case LAPLACE_P2: return launch_fwd_multi_t<2, LAPLACE_P2, JAC_COMP>(P, st);
    case ELASTIC_P1: return launch_fwd_multi_t<2, ELASTIC_P1, JAC_COMP>(P, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int FORM>
static cudaError_t bwd_form(bool saved_det, const BwdMulti& P, cudaStream_t st) {
  return saved_det ? launch_bwd_multi_t<2, FORM, JAC_SAVED>(P, st) : launch_bwd_multi_t<2, FORM, JAC_COMP>(P, st);
}

cudaError_t launch_bwd_multi_d2(int form, bool saved_det, const BwdMulti& P, cudaStream_t st) {
  switch (form) {
    case LAPLACE_P1: return bwd_form<LAPLACE_P1>(saved_det, P, st);
    case LAPLACE_P2: return bwd_form<LAPLACE_P2>(saved_det, P, st);
    case ELASTIC_P1: return bwd_form<ELASTIC_P1>(saved_det, P, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reduce_multi_d2(const RedMulti& P, cudaStream_t st) { return launch_reduce_multi_t<2>(P, st); }

}  // namespace fem
