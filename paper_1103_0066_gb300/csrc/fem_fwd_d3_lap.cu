// Forward kernels for tetrahedra, P1 and P2 Laplacian.
#include "fem_fwd.cuh"

namespace fem {
cudaError_t launch_fwd_d3_lap(const FwdLaunch& L) {
  switch (L.form) {
    case LAPLACE_P1: return launch_fwd_form<3, LAPLACE_P1>(L);
    case LAPLACE_P2: return launch_fwd_form<3, LAPLACE_P2>(L);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace fem
