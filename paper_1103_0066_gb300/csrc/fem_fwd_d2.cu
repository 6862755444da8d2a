// Forward kernels for triangles (all forms).
#include "fem_fwd.cuh"

namespace fem {
cudaError_t launch_fwd_d2(const FwdLaunch& L) {
  switch (L.form) {
    case LAPLACE_P1: return launch_fwd_form<2, LAPLACE_P1>(L);
    case LAPLACE_P2: return launch_fwd_form<2, LAPLACE_P2>(L);
    case ELASTIC_P1: return launch_fwd_form<2, ELASTIC_P1>(L);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace fem
